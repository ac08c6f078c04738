// Request engine behind dtw_submit / dtw_poll: continuous batching of
// alignments (the serving pattern built on Algorithm 2's level structure).
//
// Each (cost kind, dimension) group has its own engine: a worker thread, a
// CUDA stream and one fixed device arena.  The groups' threads run at the same
// time, so levels of different groups (say d=12 and d=64 requests) overlap on
// the device.  With an admission budget (dtw_set_budget) the arenas share it in
// proportion to the footprint of the requests each group has received (at least
// a quarter each); an idle engine whose share has drifted by more than a
// quarter gives its arena back and takes the new share at its next request.
// Each iteration of a group:
//   1. admits queued requests while a pair slot, their rows of the per-row path
//      arrays, their staging bytes and their share of the level scratch (linear
//      in M+N, Section 4.3's memory argument) are free -- requests that arrive
//      while others are in flight join here, at the next level boundary;
//   2. appends the admitted pairs' root boxes to the live box list (small ones
//      straight to the base list);
//   3. runs ONE recursion level for every box of every active pair together:
//      plan -> sweep -> split -> base cases -> plan of the next level, then
//      marks which pairs still own boxes and reads the control block back once;
//   4. finishes the pairs that own no box any more: path assembly, results
//      copied out, resources returned.
// Different requests are therefore at different recursion levels inside the
// same launches.  With DTW_SERVE_TRACE set in the environment each engine logs
// its iterations (admissions, level ends, finished tickets) to stderr.  Each box is computed exactly as in dtw_align, so a result does
// not depend on which other requests share its launches.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "dtw_b300.h"
#include "dtw_common.cuh"
#include "dtw_kernels.h"
#include "workspace.h"

using namespace dtwb;

namespace {

// First-fit allocator over the integer range [0, cap).
struct RangeAlloc {
    std::map<long long, long long> free_;  // offset -> length
    void init(long long cap) {
        free_.clear();
        if (cap > 0) free_[0] = cap;
    }
    long long alloc(long long n, long long align) {
        if (n <= 0) return 0;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            const long long o0 = it->first, end = it->first + it->second;
            const long long off = (o0 + align - 1) / align * align;
            if (off + n <= end) {
                free_.erase(it);
                if (off > o0) free_[o0] = off - o0;
                if (off + n < end) free_[off + n] = end - (off + n);
                return off;
            }
        }
        return -1;
    }
    void release(long long off, long long n) {
        if (n <= 0) return;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Pending {
    long long ticket;
    dtw_request r;
};

struct Active {
    long long ticket = -1;
    int64_t M = 0, N = 0;
    long long row_off = 0;
    long long byte_off = -1, byte_n = 0;
    int32_t* path_host = nullptr;  // caller's host path buffer (the device copy is staged)
    int32_t* path_dev = nullptr;
};

struct Result {
    int status;
    int64_t K;
    double cost;
};

constexpr int kSlots = 4096;                 // pairs in flight per group
constexpr size_t kDefaultArena = 2ull << 30;  // bytes per group when no budget is set
constexpr size_t kMinArena = 96ull << 20;     // the smallest arena an engine starts with

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

bool device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int status_of(int err) {
    switch (err) {
        case ERR_NONE: return DTW_OK;
        case ERR_TIMEOUT: return DTW_ETIMEOUT;
        case ERR_OVERFLOW: return DTW_EOVERFLOW;
        case ERR_CAPACITY: return DTW_ENOMEM;
        default: return DTW_EINTERNAL;
    }
}

struct Server;

// One (kind, d) group: its arena, its live recursion state and its active pairs.
struct Engine {
    int kind = 0, d = 1;
    cudaStream_t st = nullptr;
    char* ws = nullptr;
    size_t arena = 0;  // bytes taken from the budget (0: none)
    bool running = false;  // under the server's mutex: the engine's thread is iterating
    Layout L{};
    long long S_max = 0, S_active = 0, stage_cap = 0;
    RangeAlloc rows, bytes;
    std::vector<int> free_slots;
    std::map<int, Active> active;  // slot -> pair
    std::deque<Pending> queue;
    int n_cur = 0;
    Box *cur = nullptr, *nxt = nullptr;
    Box* d_roots = nullptr;
    int32_t *d_flags = nullptr, *d_err = nullptr, *d_idx = nullptr;
    int num_sms = 0;
    long long base_area = 16384;
    int spin_limit = 1 << 22;

    int windows = kSplitWindowsDefault;  // windows of split rows per box at most (fixed at init)

    int init(size_t arena, int sms) {
        num_sms = sms;
        windows = split_windows_option();
        // arena: level scratch (about 1.75 KB per unit of M+N) + staging bytes + fixed parts
        const size_t fixed = (size_t)kSlots * (sizeof(PairDesc) + sizeof(PairRes) + sizeof(Box) + 3 * 4 + 16) + (1 << 20);
        if (arena < fixed + (64 << 20)) arena = fixed + (64 << 20);
        const size_t stage = (arena - fixed) * 2 / 5;
        S_max = (long long)((arena - fixed - stage) / 1800);
        for (;;) {
            L = make_layout(kSlots, S_max, 0, (long long)stage, 0, windows, split_win_rows(kind));
            if (L.total + fixed <= arena || S_max < 1024) break;
            S_max = S_max * 15 / 16;
        }
        const size_t extra = up256(sizeof(Box) * kSlots) + 3 * up256(4 * kSlots);
        if (cudaMalloc(&ws, L.total + extra) != cudaSuccess) {
            cudaGetLastError();
            ws = nullptr;
            return DTW_ENOMEM;
        }
        if (!st && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return DTW_ECUDA;
        char* x = ws + L.total;
        d_roots = reinterpret_cast<Box*>(x);
        x += up256(sizeof(Box) * kSlots);
        d_flags = reinterpret_cast<int32_t*>(x);
        x += up256(4 * kSlots);
        d_err = reinterpret_cast<int32_t*>(x);
        x += up256(4 * kSlots);
        d_idx = reinterpret_cast<int32_t*>(x);
        // boundary words must not carry a future epoch; the control block starts empty
        if (cudaMemsetAsync(ws, 0, L.total, st) != cudaSuccess) return DTW_ECUDA;
        LevelCtl c0{};
        c0.epoch_base = 1;
        if (cudaMemcpyAsync(ws + L.ctl, &c0, sizeof(c0), cudaMemcpyHostToDevice, st) != cudaSuccess) return DTW_ECUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return DTW_ECUDA;
        rows.init(S_max);
        bytes.init((long long)stage);
        stage_cap = (long long)stage;
        free_slots.clear();
        for (int k = kSlots - 1; k >= 0; --k) free_slots.push_back(k);
        cur = reinterpret_cast<Box*>(ws + L.boxA);
        nxt = reinterpret_cast<Box*>(ws + L.boxB);
        return DTW_OK;
    }

    // Gives the arena back (the engine must be idle); the next request re-creates it.
    void free_arena() {
        if (!ws) return;
        cudaStreamSynchronize(st);
        cudaFree(ws);
        ws = nullptr;
        n_cur = 0;
    }

    bool idle() const { return active.empty() && queue.empty(); }
    LevelCtl* ctl() { return reinterpret_cast<LevelCtl*>(ws + L.ctl); }
    PairDesc* pairs() { return reinterpret_cast<PairDesc*>(ws + L.pairs); }
    PairRes* pres() { return reinterpret_cast<PairRes*>(ws + L.pres); }
    int32_t* jlo() { return reinterpret_cast<int32_t*>(ws + L.jlo); }
    int32_t* jhi() { return reinterpret_cast<int32_t*>(ws + L.jhi); }
    int32_t* off() { return reinterpret_cast<int32_t*>(ws + L.off); }

    void release(int slot) {
        Active& a = active[slot];
        rows.release(a.row_off, a.M);
        if (a.byte_off >= 0) bytes.release(a.byte_off, a.byte_n);
        S_active -= a.M + a.N;
        free_slots.push_back(slot);
        active.erase(slot);
    }

    // One iteration; finished requests go to `out`.
    int iterate(std::mutex& mu, std::vector<std::pair<long long, Result>>& out);
};

struct Server {
    std::mutex mu;
    std::condition_variable cv;
    std::map<std::pair<int, int>, std::unique_ptr<Engine>> engines;
    std::map<Engine*, double> demand;  // footprint of the requests each group has received
    std::unordered_map<long long, Result> done;
    std::unordered_set<long long> inflight;
    long long next_ticket = 0;
    int device = 0;
    uint64_t budget = 0;
    size_t allocated = 0;  // arena bytes taken from the budget by all engines
    size_t max_queue = 1 << 20;

    size_t target_arena(Engine* en);  // under mu
    void engine_loop(Engine* en);
};

Server& server() {
    static Server* s = new Server();  // never destroyed: the worker may outlive static destruction
    return *s;
}

static bool g_trace = getenv("DTW_SERVE_TRACE") != nullptr;
// Engines that exist.  While another engine exists, an engine's sweeps run on
// 15/16 of the SMs at most, one block per SM: a group's level of many bands would
// otherwise hold every SM with persistent blocks for the whole level (a level-0
// block holds its ticket for milliseconds), and a request of another group that
// arrives meanwhile would wait for that level to end.  Its plan kernel (1024
// threads of 64 registers) and float split kernel (256 threads of about 250)
// each need a whole SM's register file, which only an SM without a sweep block
// has; a d=64 sweep block needs most of an SM's shared memory.
static std::atomic<int> g_live_engines{0};
static double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int Engine::iterate(std::mutex& mu, std::vector<std::pair<long long, Result>>& out) {
    const size_t esize = 4;
    if (g_trace) fprintf(stderr, "[serve] %.3f kind %d d %d iterate: active %zu queue %zu n_cur %d\n", now_ms(), kind, d, active.size(), queue.size(), n_cur);
    // ---- 1. admission
    std::vector<Box> roots;
    std::vector<int> admitted;
    {
        std::lock_guard<std::mutex> g(mu);
        while (!queue.empty() && !free_slots.empty()) {
            const Pending& p = queue.front();
            const dtw_request& r = p.r;
            const bool xd = device_ptr(r.X), yd = device_ptr(r.Y), pd = device_ptr(r.path_out);
            const long long fb = (xd ? 0 : (long long)up256((size_t)r.M * r.d * esize)) +
                                 (yd ? 0 : (long long)up256((size_t)r.N * r.d * esize)) +
                                 (pd ? 0 : (long long)up256(8 * (size_t)(r.M + r.N - 1)));
            if (r.M + r.N > S_max || fb > stage_cap) {  // can never fit
                out.push_back({p.ticket, Result{DTW_ENOMEM, 0, 0.0}});
                queue.pop_front();
                continue;
            }
            if (S_active + r.M + r.N > S_max) break;
            const long long ro = rows.alloc(r.M, 1);
            if (ro < 0) break;
            const long long bo = fb > 0 ? bytes.alloc(fb, 256) : -1;
            if (fb > 0 && bo < 0) {
                rows.release(ro, r.M);
                break;
            }
            const int slot = free_slots.back();
            free_slots.pop_back();
            Active a;
            a.ticket = p.ticket;
            a.M = r.M;
            a.N = r.N;
            a.row_off = ro;
            a.byte_off = bo;
            a.byte_n = fb;
            char* stage = ws + L.feat + (bo >= 0 ? bo : 0);
            PairDesc desc{};
            desc.M = (int32_t)r.M;
            desc.N = (int32_t)r.N;
            desc.row_off = (int32_t)ro;
            cudaError_t e = cudaSuccess;
            if (xd) {
                desc.X = r.X;
            } else {
                desc.X = stage;
                e = cudaMemcpyAsync(stage, r.X, (size_t)r.M * r.d * esize, cudaMemcpyHostToDevice, st);
                stage += up256((size_t)r.M * r.d * esize);
            }
            if (yd) {
                desc.Y = r.Y;
            } else if (e == cudaSuccess) {
                desc.Y = stage;
                e = cudaMemcpyAsync(stage, r.Y, (size_t)r.N * r.d * esize, cudaMemcpyHostToDevice, st);
                stage += up256((size_t)r.N * r.d * esize);
            }
            if (pd) {
                a.path_dev = r.path_out;
            } else {
                a.path_dev = reinterpret_cast<int32_t*>(stage);
                a.path_host = r.path_out;
            }
            desc.path = a.path_dev;
            if (e == cudaSuccess) e = cudaMemcpyAsync(pairs() + slot, &desc, sizeof(desc), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = launch_fill_i32(jlo() + ro, r.M, INT32_MAX, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(jhi() + ro, 0xff, 4 * (size_t)r.M, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(pres() + slot, 0, sizeof(PairRes), st);
            if (e != cudaSuccess) return DTW_ECUDA;
            active[slot] = a;
            S_active += r.M + r.N;
            admitted.push_back(slot);
            queue.pop_front();
        }
    }
    // integer pairs: exactness guard, per pair
    if (kind == KIND_ABS && !admitted.empty()) {
        for (int slot : admitted) {
            const Active& a = active[slot];
            cudaError_t e = launch_int_range_check(pairs() + slot, 1, (int)std::max(a.M, a.N),
                                                   reinterpret_cast<int32_t*>(ws + L.minmax) + 4 * slot, ctl(), st,
                                                   d_err + slot);
            if (e != cudaSuccess) return DTW_ECUDA;
        }
        std::vector<int32_t> herr(kSlots);
        if (cudaMemcpyAsync(herr.data(), d_err, 4 * kSlots, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return DTW_ECUDA;
        std::vector<int> ok;
        for (int slot : admitted) {
            if (herr[slot]) {
                out.push_back({active[slot].ticket, Result{DTW_EOVERFLOW, 0, 0.0}});
                release(slot);
            } else {
                ok.push_back(slot);
            }
        }
        admitted.swap(ok);
    }
    int n_new_cur = 0;
    for (int slot : admitted) {
        const Active& a = active[slot];
        Box r{};
        r.pair = slot;
        r.H = (int32_t)a.M;
        r.W = (int32_t)a.N;
        r.flags = BOX_ROOT;
        r.known_i = -1;
        r.known_f = NAN;
        if (a.M * a.N > base_area) ++n_new_cur;
        roots.push_back(r);
    }
    if (!roots.empty()) {
        if (cudaMemcpyAsync(d_roots, roots.data(), sizeof(Box) * roots.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
            return DTW_ECUDA;
        if (launch_append_roots(d_roots, (int)roots.size(), cur, n_cur, reinterpret_cast<Box*>(ws + L.base),
                                (int)L.cap_base, base_area, ctl(), st) != cudaSuccess)
            return DTW_ECUDA;
        n_cur += n_new_cur;
    }
    if (active.empty()) return DTW_OK;

    // ---- 2. one level for every active pair
    const int halo = kind == KIND_ABS ? kSplitHalo : 0;
    const int U = sweep_block_cols(kind, d), BR = sweep_band_rows(kind, d), G = sweep_group_bands(kind);
    int* d_boxdone = reinterpret_cast<int*>(ws + L.boxdone);
    Sweep* d_sweeps = reinterpret_cast<Sweep*>(ws + L.sweeps);
    SweepRes* d_sres = reinterpret_cast<SweepRes*>(ws + L.sres);
    Box* d_base = reinterpret_cast<Box*>(ws + L.base);
    cudaError_t e = cudaSuccess;
    if (n_cur > 0) {
        PlanArgs pa{cur, n_cur, pairs(), MODE_ALIGN, kind, halo, U, BR, G, d_sweeps, ctl(),
                    L.cap_sweeps, L.cap_buf, L.cap_out, d_boxdone, L.cap_items, false, nullptr};
        pa.tmap = reinterpret_cast<int2*>(ws + L.tmap);
        pa.cap_tickets = L.cap_tickets;
        pa.map_min = num_sms;
        pa.nwin = windows;
        pa.whole_groups = sweep_whole_groups(kind, d);
        e = launch_plan(pa, st);
        SweepArgs sa{d_sweeps, ctl(), reinterpret_cast<unsigned long long*>(ws + L.bufpool), ws + L.outpool, d_sres,
                     d, spin_limit, -1};
        sa.tmap = reinterpret_cast<const int2*>(ws + L.tmap);
        const long long cap = g_live_engines.load(std::memory_order_relaxed) > 1 ? num_sms - num_sms / 16 : 0;
        if (e == cudaSuccess) e = launch_sweep(kind, d, kind == KIND_ABS, sa, num_sms, cap, st);
        SplitArgs sp{cur, n_cur, pairs(), pres(), kind, d, halo, d_sweeps, d_sres, ws + L.outpool, nxt, d_base,
                     ctl(), base_area, (int)L.cap_box, (int)L.cap_base, d_boxdone, ws + L.partials, -1, num_sms};
        if (e == cudaSuccess) e = launch_split(sp, st);
    }
    BaseArgs ba{d_base, -1, pairs(), pres(), jlo(), jhi(), ctl(), kind, d};
    if (e == cudaSuccess) e = launch_base(ba, st);
    PlanArgs pn{nxt, -1, pairs(), MODE_ALIGN, kind, halo, U, BR, G, d_sweeps, ctl(),
                L.cap_sweeps, L.cap_buf, L.cap_out, d_boxdone, L.cap_items, true, nullptr};
    pn.tmap = reinterpret_cast<int2*>(ws + L.tmap);
    pn.cap_tickets = L.cap_tickets;
    pn.map_min = num_sms;
    pn.nwin = windows;
    pn.whole_groups = sweep_whole_groups(kind, d);
    if (e == cudaSuccess) e = launch_plan(pn, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_flags, 0, 4 * kSlots, st);
    if (e == cudaSuccess) e = launch_mark_pairs(nxt, ctl(), d_flags, st);
    LevelCtl hc{};
    std::vector<int32_t> flags(kSlots);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, ctl(), sizeof(hc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(flags.data(), d_flags, 4 * kSlots, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return DTW_ECUDA;
    std::swap(cur, nxt);
    n_cur = hc.n_cur;
    if (hc.err != ERR_NONE) return status_of(hc.err);

    if (g_trace) fprintf(stderr, "[serve] %.3f kind %d level done: n_cur %d n_base %d\n", now_ms(), kind, hc.n_cur, hc.n_base);
    // ---- 3. pairs that own no box any more are complete
    std::vector<int> fin;
    int max_M = 1;
    for (auto& kv : active) {
        if (!flags[kv.first]) {
            fin.push_back(kv.first);
            max_M = std::max<int>(max_M, (int)kv.second.M);
        }
    }
    if (fin.empty()) return DTW_OK;
    e = cudaMemcpyAsync(d_idx, fin.data(), 4 * fin.size(), cudaMemcpyHostToDevice, st);
    AssembleArgs aa{pairs(), (int)fin.size(), max_M, pres(), jlo(), jhi(), off(), ctl(), d_idx};
    if (e == cudaSuccess) e = launch_assemble(aa, st);
    std::vector<PairRes> pr(fin.size());
    for (size_t k = 0; k < fin.size() && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(&pr[k], pres() + fin[k], sizeof(PairRes), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, ctl(), sizeof(hc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return DTW_ECUDA;
    if (hc.err != ERR_NONE) return status_of(hc.err);
    for (size_t k = 0; k < fin.size() && e == cudaSuccess; ++k) {
        const Active& a = active[fin[k]];
        if (a.path_host)
            e = cudaMemcpyAsync(a.path_host, a.path_dev, sizeof(int32_t) * 2 * (size_t)pr[k].K,
                                cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return DTW_ECUDA;
    for (size_t k = 0; k < fin.size(); ++k) {
        const Active& a = active[fin[k]];
        if (g_trace) fprintf(stderr, "[serve] %.3f kind %d finished ticket %lld\n", now_ms(), kind, a.ticket);
        const double cost = kind == KIND_ABS ? (double)pr[k].cost_i : pr[k].cost_f;
        out.push_back({a.ticket, Result{DTW_OK, pr[k].K, cost}});
        release(fin[k]);
    }
    return DTW_OK;
}

// The engine's share of the budget: its groups' part of the footprint received
// so far, at least a quarter (a second group always finds room).
size_t Server::target_arena(Engine* en) {
    if (!budget) return kDefaultArena;
    double tot = 0;
    for (auto& kv : demand) tot += kv.second;
    double share = tot > 0 ? demand[en] / tot : 1.0;
    if (engines.size() > 1) share = std::min(std::max(share, 0.25), 0.75);
    return (size_t)(share * (double)budget);
}

void Server::engine_loop(Engine* en) {
    cudaSetDevice(device);
    for (;;) {
        size_t arena = 0;
        {
            std::unique_lock<std::mutex> g(mu);
            cv.wait(g, [&] { return !en->idle(); });
            en->running = true;
            if (!en->ws) {
                // take the engine's share of what the budget has left; wait while
                // another engine still holds more than its share
                for (;;) {
                    const size_t want = target_arena(en);
                    size_t left = budget ? (budget > allocated ? budget - allocated : 0) : want;
                    if (budget && left < want) {
                        // idle engines holding more than their share give it back
                        // (their threads wait for work and re-check their arena)
                        for (auto& kv : engines) {
                            Engine* o = kv.second.get();
                            if (o != en && !o->running && o->ws && o->idle() && o->arena > target_arena(o)) {
                                o->free_arena();
                                allocated -= o->arena;
                                o->arena = 0;
                            }
                        }
                        left = budget > allocated ? budget - allocated : 0;
                    }
                    arena = std::min(want, left);
                    if (!budget || arena >= std::min<size_t>(want, kMinArena)) break;
                    cv.wait_for(g, std::chrono::milliseconds(1));
                }
                if (budget) allocated += arena;
            }
        }
        if (!en->ws) {
            int sms = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
            int rc = en->init(arena, sms);
            if (rc == DTW_OK) {
                en->arena = arena;
            } else {
                if (en->ws) cudaFree(en->ws);
                en->ws = nullptr;
                std::lock_guard<std::mutex> g(mu);
                if (budget) allocated -= arena;
                for (const Pending& p : en->queue) {
                    done[p.ticket] = Result{rc, 0, 0.0};
                    inflight.erase(p.ticket);
                }
                en->queue.clear();
                en->running = false;
                continue;
            }
        }
        std::vector<std::pair<long long, Result>> out;
        const int rc = en->iterate(mu, out);
        if (rc != DTW_OK) {
            // a device-side error or a failed CUDA call poisons the group's
            // in-flight state: fail its active pairs and start it afresh
            for (auto& kv : en->active) out.push_back({kv.second.ticket, Result{rc, 0, 0.0}});
            std::vector<int> slots;
            for (auto& kv : en->active) slots.push_back(kv.first);
            for (int sl : slots) en->release(sl);
            en->n_cur = 0;
            cudaGetLastError();
            LevelCtl c0{};
            LevelCtl old{};
            cudaMemcpyAsync(&old, en->ctl(), sizeof(old), cudaMemcpyDeviceToHost, en->st);
            cudaStreamSynchronize(en->st);
            c0.epoch_base = old.epoch_base + 1;
            cudaMemcpyAsync(en->ctl(), &c0, sizeof(c0), cudaMemcpyHostToDevice, en->st);
            cudaStreamSynchronize(en->st);
        }
        std::lock_guard<std::mutex> g(mu);
        for (auto& r : out) {
            done[r.first] = r.second;
            inflight.erase(r.first);
        }
        en->running = false;
        if (budget && en->ws && en->idle()) {
            // an idle engine whose share has drifted gives its arena back
            const double want = (double)target_arena(en), have = (double)en->arena;
            if (want > 1.25 * have || want < 0.75 * have) {
                en->free_arena();
                allocated -= en->arena;
                en->arena = 0;
                cv.notify_all();
            }
        }
    }
}

}  // namespace

extern "C" {

int64_t dtw_submit(const dtw_request* r) {
    if (!r || !r->X || !r->Y || !r->path_out || r->M < 1 || r->N < 1 || r->d < 1) return DTW_EINVAL;
    const int k = r->cost_kind & 0xff, flags = r->cost_kind & ~0xff;
    if (k != DTW_EUCLID_F32 && k != DTW_ABS_I32) return DTW_EINVAL;
    // forms: the compensated FP32 DP and the BF16 tensor-core cost (the plain FP64 form is not served)
    if (flags & ~(int)(DTW_DP_F32_KAHAN | DTW_COST_BF16)) return DTW_EINVAL;
    if (flags && k != DTW_EUCLID_F32) return DTW_EINVAL;
    if ((flags & DTW_COST_BF16) && r->d != 64) return DTW_EINVAL;
    if (k == DTW_ABS_I32 && r->d != 1) return DTW_EINVAL;
    if (r->M > (1LL << 30) || r->N > (1LL << 30)) return DTW_EINVAL;
    const int kind = k == DTW_ABS_I32 ? KIND_ABS
                                      : ((flags & DTW_COST_BF16) ? KIND_EUCB
                                                                 : ((flags & DTW_DP_F32_KAHAN) ? KIND_EUCF : KIND_EUC));
    if (kind != KIND_ABS && (r->d == 12 || r->d == 64) &&
        ((reinterpret_cast<uintptr_t>(r->X) | reinterpret_cast<uintptr_t>(r->Y)) & 15))
        return DTW_EINVAL;  // the d=12 kernels load frames in 16-byte pieces
    Server& s = server();
    std::lock_guard<std::mutex> g(s.mu);
    if (s.inflight.size() >= s.max_queue) return DTW_EBUSY;
    if (s.engines.empty() && cudaGetDevice(&s.device) != cudaSuccess) return DTW_ECUDA;
    auto key = std::make_pair(kind, kind == KIND_ABS ? 1 : (int)r->d);
    auto& en = s.engines[key];
    if (!en) {
        en.reset(new Engine());
        en->kind = kind;
        en->d = key.second;
        s.demand[en.get()] = 0.0;
        g_live_engines.fetch_add(1);
        std::thread(&Server::engine_loop, &s, en.get()).detach();
    }
    // the group's demand: level scratch and features, linear in M + N
    s.demand[en.get()] += (double)(r->M + r->N) * (1800.0 + 4.0 * (double)r->d);
    const long long t = s.next_ticket++;
    en->queue.push_back(Pending{t, *r});
    s.inflight.insert(t);
    s.cv.notify_all();
    return t;
}

int dtw_poll(int64_t ticket, int64_t* K_out, double* cost_out) {
    Server& s = server();
    std::lock_guard<std::mutex> g(s.mu);
    auto it = s.done.find(ticket);
    if (it == s.done.end()) return s.inflight.count(ticket) ? DTW_PENDING : DTW_EINVAL;
    const Result r = it->second;
    s.done.erase(it);
    if (K_out) *K_out = r.K;
    if (cost_out) *cost_out = r.cost;
    return r.status;
}

}  // extern "C"

namespace dtwb {
void serve_set_budget(uint64_t bytes) {
    Server& s = server();
    std::lock_guard<std::mutex> g(s.mu);
    s.budget = bytes;
}
}  // namespace dtwb
