// C ABI of the library: argument checks, workspace, staging of host buffers,
// and the host side of the level loop of Algorithm 2 (Section 3.2).  The device
// does all the arithmetic.  The level loop (plan -> sweep -> split per level)
// runs as one CUDA graph whose continuation the device decides, or, with
// per-level timing or DTW_OPT_GRAPH = 0, from the host, which then reads back one
// small control block per level to learn whether another level exists.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "dtw_b300.h"
#include "dtw_common.cuh"
#include "dtw_kernels.h"
#include "workspace.h"

using namespace dtwb;

namespace {

struct Ctx {
    std::mutex mu;
    cudaStream_t stream = nullptr;
    uint64_t budget = 0;
    void* arena = nullptr;
    uint64_t arena_bytes = 0;
    void* ws = nullptr;  // library-owned workspace
    size_t ws_bytes = 0;
    int timing = 0;
    long long base_area = 16384;
    int spin_limit = 1 << 22;
    int fused_split = 1;  // the split in the sweep kernel: 0 never, 1 float kinds and batches, 2 always (not BF16)
    int split_windows = kSplitWindowsDefault;  // windows of split rows per box at most
    long long skip_publish = -1;
    uint32_t epoch = 1;  // next boundary-word epoch; increases across calls
    int num_sms = 0;
    int device = -1;
    dtw_stats stats = {};
    int use_graph = 1;
    int variant = 0;  // integer sweep variant (rows per lane), see sweep_band_rows
    int32_t esub = 1, egap = 1;  // edit distance: substitution and gap costs
    int32_t ematch = 0;          // and the match cost (local alignment's passes set it negative)
    // cached executable graph of the level loop and the parameters it was built for
    struct LevelGraph {
        cudaGraphExec_t exec = nullptr;
        cudaStream_t cap = nullptr;  // capture stream (the library stream may be the legacy one)
        std::vector<long long> key;
    } lg;
};

Ctx& ctx() {
    static Ctx c;
    return c;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int ensure_device(Ctx& c) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DTW_ECUDA;
    if (dev != c.device || c.num_sms == 0) {
        if (cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return DTW_ECUDA;
        if (c.ws) {
            cudaFree(c.ws);
            c.ws = nullptr;
            c.ws_bytes = 0;
        }
        c.device = dev;
    }
    return DTW_OK;
}

// Returns a device workspace of at least `bytes` (the arena or a cached cudaMalloc).
int workspace(Ctx& c, size_t bytes, void** out) {
    if (c.budget && bytes > c.budget) return DTW_ENOMEM;
    if (c.arena) {
        if (bytes > c.arena_bytes) return DTW_ENOMEM;
        *out = c.arena;
        return DTW_OK;
    }
    if (c.ws_bytes < bytes) {
        if (c.ws) {
            cudaStreamSynchronize(c.stream);
            cudaFree(c.ws);
            c.ws = nullptr;
            c.ws_bytes = 0;
        }
        const size_t want = bytes + bytes / 4;
        if (cudaMalloc(&c.ws, want) != cudaSuccess) {
            cudaGetLastError();
            return DTW_ENOMEM;
        }
        // boundary words must not carry a future epoch by accident
        if (cudaMemsetAsync(c.ws, 0, want, c.stream) != cudaSuccess) return DTW_ECUDA;
        c.ws_bytes = want;
    }
    *out = c.ws;
    return DTW_OK;
}

// The level loop of Algorithm 2 as one CUDA graph: a WHILE node whose body is
// sweep -> split -> plan of the next level (which copies the next boxes into the
// current list) -> condition kernel.  No host round trip per level.
int level_graph(Ctx& c, const std::vector<long long>& key, const SweepArgs& sa, const SplitArgs& sp,
                const PlanArgs& pn, LevelCtl* ctl, int kind, int d, int variant, int max_levels, cudaGraphExec_t* out) {
    auto& lg = c.lg;
    if (lg.exec && lg.key == key) {
        *out = lg.exec;
        return DTW_OK;
    }
    if (lg.exec) {
        cudaGraphExecDestroy(lg.exec);
        lg.exec = nullptr;
    }
    if (!lg.cap && cudaStreamCreateWithFlags(&lg.cap, cudaStreamNonBlocking) != cudaSuccess) return DTW_ECUDA;
    // integer kinds: two sweep kernels, with and without tagged sweeps (the
    // latter holds fewer registers, so more blocks fit an SM), chosen per level
    const bool two = int_kind(kind);
    if (sweep_prepare(kind, d, int_kind(kind), variant) != cudaSuccess) return DTW_ECUDA;
    if (two && sweep_prepare(kind, d, false, variant) != cudaSuccess) return DTW_ECUDA;
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return DTW_ECUDA;
    int rc = DTW_OK;
    cudaGraphConditionalHandle h;
    cudaGraphNodeParams np{};
    cudaGraphNode_t node;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    }
    if (e == cudaSuccess) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        cudaGraphNode_t last = nullptr;  // the body's node the split and plan follow
        if (two) {
            // body: select -> IF(no tagged box) { sweep } -> IF(tagged boxes) { sweep with tags } -> ...
            cudaGraphConditionalHandle hk[2];
            for (int k = 0; k < 2 && e == cudaSuccess; ++k)
                e = cudaGraphConditionalHandleCreate(&hk[k], body, 0, 0);
            if (e == cudaSuccess)
                e = cudaStreamBeginCaptureToGraph(lg.cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e1 = launch_sweep_select(ctl, hk[0], hk[1], lg.cap);
                const cudaGraphNode_t* deps = nullptr;
                size_t ndeps = 0;
                cudaStreamCaptureStatus cs;
                if (e1 == cudaSuccess) e1 = cudaStreamGetCaptureInfo(lg.cap, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
                if (e1 == cudaSuccess && ndeps == 1) last = deps[0];
                else if (e1 == cudaSuccess) e1 = cudaErrorUnknown;
                cudaGraph_t got = nullptr;
                e = cudaStreamEndCapture(lg.cap, &got);
                if (e == cudaSuccess) e = e1;
            }
            for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
                cudaGraphNodeParams ip{};
                ip.type = cudaGraphNodeTypeConditional;
                ip.conditional.handle = hk[k];
                ip.conditional.type = cudaGraphCondTypeIf;
                ip.conditional.size = 1;
                cudaGraphNode_t inode;
                e = cudaGraphAddNode(&inode, body, &last, nullptr, 1, &ip);
                if (e != cudaSuccess) break;
                e = cudaStreamBeginCaptureToGraph(lg.cap, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaError_t e1 = launch_sweep(kind, d, k == 1, sa, c.num_sms, 0, lg.cap, variant);
                    cudaGraph_t got = nullptr;
                    e = cudaStreamEndCapture(lg.cap, &got);
                    if (e == cudaSuccess) e = e1;
                }
                last = inode;
            }
        }
        if (e == cudaSuccess)
            e = cudaStreamBeginCaptureToGraph(lg.cap, body, last ? &last : nullptr, nullptr, last ? 1 : 0,
                                              cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = two ? cudaSuccess : launch_sweep(kind, d, false, sa, c.num_sms, 0, lg.cap, variant);
            if (e1 == cudaSuccess && sa.prog == nullptr) e1 = launch_split(sp, lg.cap);
            if (e1 == cudaSuccess) e1 = launch_plan(pn, lg.cap);
            if (e1 == cudaSuccess) e1 = launch_level_cond(ctl, h, max_levels, lg.cap);
            cudaGraph_t got = nullptr;
            e = cudaStreamEndCapture(lg.cap, &got);
            if (e == cudaSuccess) e = e1;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&lg.exec, g, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        lg.exec = nullptr;
        rc = DTW_ECUDA;
    } else {
        lg.key = key;
        *out = lg.exec;
    }
    cudaGraphDestroy(g);
    return rc;
}

int map_device_error(int err) {
    switch (err) {
        case ERR_NONE: return DTW_OK;
        case ERR_TIMEOUT: return DTW_ETIMEOUT;
        case ERR_OVERFLOW: return DTW_EOVERFLOW;
        case ERR_CAPACITY: return DTW_ENOMEM;
        default: return DTW_EINTERNAL;
    }
}

int check_kind(int32_t cost_kind, int32_t d, int* kind, bool* plain) {
    const int k = cost_kind & 0xff;
    const int flags = cost_kind & ~0xff;
    if (k == DTW_EDIT_I32) {  // no forms, no plain comparator; one symbol per frame
        if (flags || d != 1) return DTW_EINVAL;
        *kind = KIND_EDIT;
        *plain = false;
        return DTW_OK;
    }
    if (k != DTW_EUCLID_F32 && k != DTW_ABS_I32) return DTW_EINVAL;
    if (flags & ~(int)(DTW_PLAIN_F64 | DTW_DP_F32_KAHAN | DTW_COST_BF16)) return DTW_EINVAL;
    if ((flags & (DTW_DP_F32_KAHAN | DTW_COST_BF16)) && (k != DTW_EUCLID_F32 || (flags & DTW_PLAIN_F64)))
        return DTW_EINVAL;
    if ((flags & DTW_COST_BF16) && d != 64) return DTW_EINVAL;  // the tensor-core tiles are built for d = 64
    if (d < 1 || (k == DTW_ABS_I32 && d != 1)) return DTW_EINVAL;
    *kind = k == DTW_ABS_I32 ? KIND_ABS
                             : ((flags & DTW_COST_BF16) ? KIND_EUCB : ((flags & DTW_DP_F32_KAHAN) ? KIND_EUCF : KIND_EUC));
    *plain = (flags & DTW_PLAIN_F64) != 0;
    return DTW_OK;
}

struct Timer {
    bool on;
    cudaStream_t st;
    std::vector<cudaEvent_t> ev;
    cudaEvent_t mark() {
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, st);
        ev.push_back(e);
        return e;
    }
    ~Timer() {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

// The tiled path for a batch.  want_path == false: dtw_cost (one full sweep).
int run_batch(Ctx& c, int B, const void* const* X, const int64_t* M, const void* const* Y, const int64_t* N, int d,
              int kind, bool want_path, int32_t* const* path_out, int64_t* K_out, double* cost_out) {
    const size_t esize = 4;  // float or int32
    long long sumM = 0, sumN = 0, feat_bytes = 0, path_pairs = 0, maxM = 0, maxN = 0;
    std::vector<char> xdev(B), ydev(B), pdev(B);
    // edit distance runs on its node grid: M+1 x N+1 nodes over the sequences
    // with a sentinel at both ends (staged into the workspace for every input)
    const bool edit = kind == KIND_EDIT;
    const int64_t* M0 = M;
    const int64_t* N0 = N;
    std::vector<int64_t> Mv, Nv;
    if (edit) {
        for (int b = 0; b < B; ++b) {
            if (M[b] < 1 || N[b] < 1 || M[b] >= (1LL << 30) || N[b] >= (1LL << 30)) return DTW_EINVAL;
            // exact int32 accumulation: every node value is at most (M+N) max(sub, gap) plus a corner term
            const long long cmax = std::max<long long>(std::max(c.esub, c.egap), std::llabs((long long)c.ematch));
            if ((M[b] + N[b] + 2) * cmax >= (1LL << 29)) return DTW_EOVERFLOW;
            Mv.push_back(M[b] + 1);
            Nv.push_back(N[b] + 1);
        }
        M = Mv.data();
        N = Nv.data();
    }
    for (int b = 0; b < B; ++b) {
        if (!X[b] || !Y[b] || M[b] < 1 || N[b] < 1 || M[b] > (1LL << 30) || N[b] > (1LL << 30)) return DTW_EINVAL;
        if (B > 65535) return DTW_EINVAL;
        if (want_path && !path_out[b]) return DTW_EINVAL;
        sumM += M[b];
        sumN += N[b];
        maxM = std::max<long long>(maxM, M[b]);
        maxN = std::max<long long>(maxN, N[b]);
        xdev[b] = is_device_ptr(X[b]);
        ydev[b] = is_device_ptr(Y[b]);
        if (edit) {
            feat_bytes += align_up((size_t)(M[b] + 1) * esize) + align_up((size_t)(N[b] + 1) * esize);
        } else {
            if (!xdev[b]) feat_bytes += align_up((size_t)M[b] * d * esize);
            if (!ydev[b]) feat_bytes += align_up((size_t)N[b] * d * esize);
        }
        if (want_path) {
            pdev[b] = is_device_ptr(path_out[b]);
            if (!pdev[b]) path_pairs += M[b] + N[b] - 1;
        }
    }
    const Layout L = make_layout(B, sumM, sumN, feat_bytes, path_pairs, c.split_windows, split_win_rows(kind));
    void* wsv = nullptr;
    int rc = workspace(c, L.total, &wsv);
    if (rc) return rc;
    char* ws = static_cast<char*>(wsv);
    cudaStream_t st = c.stream;
    Timer T{c.timing != 0, st, {}};
    cudaEvent_t t_begin = c.timing ? T.mark() : nullptr;

    // stage host features and describe the pairs
    std::vector<PairDesc> pd(B);
    size_t fo = L.feat;
    long long row_off = 0, path_off = 0;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < B && e == cudaSuccess; ++b) {
        PairDesc& p = pd[b];
        p.M = (int32_t)M[b];
        p.N = (int32_t)N[b];
        p.row_off = (int32_t)row_off;
        p.flags = 0;
        p.esub = c.esub;
        p.egap = c.egap;
        p.ematch = c.ematch;
        row_off += M[b];
        if (edit) {
            // [pad, symbols..., pad] for X and for Y
            const void* src[2] = {X[b], Y[b]};
            const int64_t len[2] = {M0[b], N0[b]};
            const bool dev[2] = {xdev[b] != 0, ydev[b] != 0};
            for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
                int32_t* dst = reinterpret_cast<int32_t*>(ws + fo);
                e = launch_fill_i32(dst, len[k] + 2, kEditPad, st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(dst + 1, src[k], (size_t)len[k] * esize,
                                        dev[k] ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
                if (k == 0) p.X = dst;
                else p.Y = dst;
                fo += align_up((size_t)(len[k] + 2) * esize);
            }
        } else if (xdev[b]) {
            p.X = X[b];
        } else {
            p.X = ws + fo;
            e = cudaMemcpyAsync(ws + fo, X[b], (size_t)M[b] * d * esize, cudaMemcpyHostToDevice, st);
            fo += align_up((size_t)M[b] * d * esize);
        }
        if (edit) {
        } else if (e == cudaSuccess && !ydev[b]) {
            p.Y = ws + fo;
            e = cudaMemcpyAsync(ws + fo, Y[b], (size_t)N[b] * d * esize, cudaMemcpyHostToDevice, st);
            fo += align_up((size_t)N[b] * d * esize);
        } else if (ydev[b]) {
            p.Y = Y[b];
        }
        if (want_path) {
            if (pdev[b]) {
                p.path = path_out[b];
            } else {
                p.path = reinterpret_cast<int32_t*>(ws + L.path) + 2 * path_off;
                path_off += M[b] + N[b] - 1;
            }
        } else {
            p.path = nullptr;
        }
    }
    if (e != cudaSuccess) return DTW_ECUDA;
    for (int b = 0; b < B; ++b) {
        if (kind != KIND_ABS && (d == 12 || d == 64) &&
            ((reinterpret_cast<uintptr_t>(pd[b].X) | reinterpret_cast<uintptr_t>(pd[b].Y)) & 15))
            return DTW_EINVAL;  // the d=12 and d=64 kernels load frames in 16-byte pieces
    }

    PairDesc* d_pairs = reinterpret_cast<PairDesc*>(ws + L.pairs);
    PairRes* d_pres = reinterpret_cast<PairRes*>(ws + L.pres);
    Box* boxA = reinterpret_cast<Box*>(ws + L.boxA);
    Box* boxB = reinterpret_cast<Box*>(ws + L.boxB);
    Box* d_base = reinterpret_cast<Box*>(ws + L.base);
    Sweep* d_sweeps = reinterpret_cast<Sweep*>(ws + L.sweeps);
    SweepRes* d_sres = reinterpret_cast<SweepRes*>(ws + L.sres);
    LevelCtl* d_ctl = reinterpret_cast<LevelCtl*>(ws + L.ctl);
    int32_t* d_jlo = reinterpret_cast<int32_t*>(ws + L.jlo);
    int32_t* d_jhi = reinterpret_cast<int32_t*>(ws + L.jhi);
    int32_t* d_off = reinterpret_cast<int32_t*>(ws + L.off);

    // root boxes: small ones go straight to the base case
    const long long base_area = want_path ? c.base_area : 0;
    std::vector<Box> roots, base_roots;
    for (int b = 0; b < B; ++b) {
        Box r{};
        r.pair = b;
        r.i0 = 0;
        r.j0 = 0;
        r.H = (int32_t)M[b];
        r.W = (int32_t)N[b];
        r.flags = BOX_ROOT;
        r.known_i = -1;
        r.known_f = NAN;
        if (want_path && M[b] * N[b] <= base_area) base_roots.push_back(r);
        else roots.push_back(r);
    }
    LevelCtl ctl0{};
    ctl0.n_base = (int32_t)base_roots.size();
    ctl0.epoch_base = c.epoch;
    e = cudaMemcpyAsync(d_pairs, pd.data(), sizeof(PairDesc) * B, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !roots.empty())
        e = cudaMemcpyAsync(boxA, roots.data(), sizeof(Box) * roots.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !base_roots.empty())
        e = cudaMemcpyAsync(d_base, base_roots.data(), sizeof(Box) * base_roots.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ctl, &ctl0, sizeof(LevelCtl), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_pres, 0, sizeof(PairRes) * B, st);
    // only this call's boundary words may bear this call's epochs
    if (e == cudaSuccess) e = cudaMemsetAsync(ws + L.bufpool, 0, 8 * (size_t)L.cap_buf, st);
    if (e == cudaSuccess && want_path) {
        e = launch_fill_i32(d_jlo, sumM, INT32_MAX, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_jhi, 0xff, 4 * (size_t)sumM, st);
    }
    if (e == cudaSuccess && kind == KIND_ABS)
        e = launch_int_range_check(d_pairs, B, (int)std::max(maxM, maxN), reinterpret_cast<int32_t*>(ws + L.minmax),
                                   d_ctl, st);
    if (e != cudaSuccess) return DTW_ECUDA;

    // ---- the level loop (Algorithm 2, breadth first: all boxes of a level together)
    // Per level: sweep -> split -> plan of the next level, then one read-back of
    // the control block (errors, the next level's box and ticket counts, which
    // size the next sweep's grid).
    const int mode = want_path ? MODE_ALIGN : MODE_COST;
    const int halo = int_kind(kind) ? kSplitHalo : 0;
    const int U = sweep_block_cols(kind, d, c.variant);
    const int BR = sweep_band_rows(kind, d, c.variant);
    const int G = sweep_group_bands(kind);
    // the first level's tickets (two half sweeps of a root box's longer side)
    // choose between the sweep's latency and throughput forms
    long long tickets0 = 0;
    for (const Box& r : roots) {
        const long long half = (std::max(r.H, r.W) + 1) / 2;
        tickets0 += 2 * (((half + BR - 1) / BR + G - 1) / G);
    }
    const int sv = sweep_variant_for(kind, d, c.variant, tickets0, c.num_sms);
    Box* cur = boxA;
    Box* nxt = boxB;
    int levels = 0, sweeps = 0;
    double sweep_ms = 0;
    LevelCtl hc = ctl0;
    // every level shrinks each box's longer side to at most about half, so the
    // depth is bounded by twice the bits of the longest sequence
    int launches = (want_path ? 1 : 0) + (kind == KIND_ABS ? 3 : 0) + (edit ? 2 * B : 0);
    const int max_levels = 2 * (64 - __builtin_clzll((unsigned long long)std::max(maxM, sumN) + 1)) + 8;
    int* d_boxdone = reinterpret_cast<int*>(ws + L.boxdone);
    int2* d_tmap = reinterpret_cast<int2*>(ws + L.tmap);
    // The graph runs the level loop on the device: it needs no level counters on
    // the host, so the root plan is not read back (no host round trip before the
    // first sweep); an error the plan records stops the loop on the device and is
    // returned from the counters read after the base case.
    const bool graph = c.use_graph && !c.timing && mode == MODE_ALIGN && !roots.empty();
    // fused split: the sweep kernel runs the level's split items once its tickets are gone
    // (default: float kinds and batches; a single integer pair keeps the separate
    // launch, measured 2% faster for it, while the 256-pair integer batch gains 14%)
    const bool fuse = mode == MODE_ALIGN && kind != KIND_EUCB &&
                      (c.fused_split == 2 || (c.fused_split == 1 && (!int_kind(kind) || B > 1)));
    int* d_prog = fuse ? reinterpret_cast<int*>(ws + L.prog) : nullptr;
    if (!roots.empty()) {
        PlanArgs pa{cur, (int)roots.size(), d_pairs, mode, kind, halo, U, BR, G, d_sweeps, d_ctl,
                    L.cap_sweeps, L.cap_buf, L.cap_out, d_boxdone, L.cap_items, false, nullptr};
        pa.tmap = d_tmap;
        pa.prog = d_prog;
        pa.nwin = c.split_windows;
        pa.whole_groups = sweep_whole_groups(kind, d);
        pa.cap_tickets = L.cap_tickets;
        pa.map_min = c.num_sms;
        e = launch_plan(pa, st);
        ++launches;
        if (!graph) {
            if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, d_ctl, sizeof(LevelCtl), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
        if (e != cudaSuccess) return DTW_ECUDA;
        if (!graph) c.epoch = hc.epoch_base;
    } else {
        hc.n_cur = 0;
    }
    if (graph) {
        SweepArgs sa{d_sweeps, d_ctl, reinterpret_cast<unsigned long long*>(ws + L.bufpool), ws + L.outpool, d_sres, d,
                     c.spin_limit, c.skip_publish};
        sa.tmap = d_tmap;
        SplitArgs sp{cur,       -1,   d_pairs, d_pres, kind,     d,          halo,    d_sweeps,
                     d_sres,    ws + L.outpool, nxt, d_base,  d_ctl,      base_area, (int)L.cap_box,
                     (int)L.cap_base, d_boxdone, ws + L.partials, -1, c.num_sms};
        PlanArgs pn{nxt, -1, d_pairs, mode, kind, halo, U, BR, G, d_sweeps, d_ctl,
                    L.cap_sweeps, L.cap_buf, L.cap_out, d_boxdone, L.cap_items, false, cur};
        pn.tmap = d_tmap;
        pn.cap_tickets = L.cap_tickets;
        pn.map_min = c.num_sms;
        pn.prog = d_prog;
        pn.nwin = c.split_windows;
        pn.whole_groups = sweep_whole_groups(kind, d);
        sa.prog = d_prog;
        sa.split = sp;
        const std::vector<long long> key{(long long)(uintptr_t)ws, (long long)L.total, L.cap_box, L.cap_base,
                                         L.cap_sweeps, L.cap_buf, L.cap_out, L.cap_items, kind, d, base_area,
                                         c.spin_limit, c.skip_publish, c.num_sms, max_levels, (long long)L.ctl,
                                         sv, d_prog != nullptr, c.split_windows};
        cudaGraphExec_t ex = nullptr;
        int grc = level_graph(c, key, sa, sp, pn, d_ctl, kind, d, sv, max_levels, &ex);
        if (grc != DTW_OK) return grc;
        if (cudaGraphLaunch(ex, st) != cudaSuccess) return DTW_ECUDA;
        hc.n_cur = 0;  // the loop ran on the device; its counters are read after the base case
        hc.n_base = -1;
    }
    while (!graph && hc.err == ERR_NONE && hc.n_cur > 0) {
        if (levels >= max_levels) return DTW_EINTERNAL;
        const int n_cur = hc.n_cur;
        SweepArgs sa{d_sweeps, d_ctl,        reinterpret_cast<unsigned long long*>(ws + L.bufpool),
                     ws + L.outpool, d_sres, d, c.spin_limit, c.skip_publish};
        sa.tmap = d_tmap;
        SplitArgs sp{cur,    n_cur,          d_pairs, d_pres, kind,      d,
                     halo,   d_sweeps,       d_sres,  ws + L.outpool, nxt, d_base,
                     d_ctl,  base_area,      (int)L.cap_box, (int)L.cap_base,
                     d_boxdone, ws + L.partials, hc.n_items, c.num_sms};
        if (d_prog != nullptr) {
            sa.prog = d_prog;
            sa.split = sp;
        }
        cudaEvent_t s0 = nullptr, s1 = nullptr;
        if (c.timing) s0 = T.mark();
        // integer levels may mix tagged and untagged boxes
        // integer kinds: the kernel with tagged sweeps only for a level that has tagged boxes
        e = launch_sweep(kind, d, mode == MODE_ALIGN && int_kind(kind) && hc.n_tag > 0, sa, c.num_sms, hc.n_tickets,
                         st, sv);
        ++launches;
        if (c.timing) s1 = T.mark();
        ++sweeps;
        if (e == cudaSuccess && mode != MODE_COST) {
            if (d_prog == nullptr) {
                e = launch_split(sp, st);
                ++launches;
            }
            // plan the next level from the boxes the split appended (count read on the device)
            PlanArgs pa{nxt, -1, d_pairs, mode, kind, halo, U, BR, G, d_sweeps, d_ctl,
                        L.cap_sweeps, L.cap_buf, L.cap_out, d_boxdone, L.cap_items, false, nullptr};
            pa.tmap = d_tmap;
            pa.prog = d_prog;
            pa.nwin = c.split_windows;
            pa.whole_groups = sweep_whole_groups(kind, d);
            pa.cap_tickets = L.cap_tickets;
            pa.map_min = c.num_sms;
            if (e == cudaSuccess) e = launch_plan(pa, st);
            ++launches;
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, d_ctl, sizeof(LevelCtl), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return DTW_ECUDA;
        c.epoch = hc.epoch_base;
        if (c.timing) sweep_ms += elapsed(s0, s1);
        ++levels;
        if (mode == MODE_COST) break;
        std::swap(cur, nxt);
    }
    if (hc.err == ERR_NONE && mode == MODE_COST) {
        std::vector<SweepRes> sr(B);
        e = cudaMemcpyAsync(sr.data(), d_sres, sizeof(SweepRes) * B, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return DTW_ECUDA;
        for (int b = 0; b < B; ++b) cost_out[b] = int_kind(kind) ? (double)sr[b].end_i : sr[b].end_f;
    }
    if (hc.err == ERR_NONE && want_path) {
        BaseArgs ba{d_base, hc.n_base, d_pairs, d_pres, d_jlo, d_jhi, d_ctl, kind, d};
        e = launch_base(ba, st);
        AssembleArgs aa{d_pairs, B, (int)maxM, d_pres, d_jlo, d_jhi, d_off, d_ctl, nullptr};
        if (e == cudaSuccess) e = launch_assemble(aa, st);
        launches += (hc.n_base != 0 ? 1 : 0) + 2;
        std::vector<PairRes> pr(B);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pr.data(), d_pres, sizeof(PairRes) * B, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, d_ctl, sizeof(LevelCtl), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return DTW_ECUDA;
        if (hc.err == ERR_NONE) {
            for (int b = 0; b < B && e == cudaSuccess; ++b) {
                K_out[b] = pr[b].K;
                cost_out[b] = int_kind(kind) ? (double)pr[b].cost_i : pr[b].cost_f;
                if (!pdev[b])
                    e = cudaMemcpyAsync(path_out[b], pd[b].path, sizeof(int32_t) * 2 * (size_t)pr[b].K,
                                        cudaMemcpyDeviceToHost, st);
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return DTW_ECUDA;
        }
    }
    if (graph) {
        c.epoch = hc.epoch_base;
        levels = sweeps = hc.levels;
        launches += 4 * hc.levels;
        if (hc.err == ERR_NONE && hc.n_cur > 0) return DTW_EINTERNAL;  // the level bound was reached
    }
    double total_ms = 0;
    if (c.timing) {
        cudaEvent_t t_end = T.mark();
        cudaEventSynchronize(t_end);
        total_ms = elapsed(t_begin, t_end);
    }
    dtw_stats& s = c.stats;
    s = dtw_stats{};
    for (int b = 0; b < B; ++b) s.problem_cells += M0[b] * N0[b];
    s.sweep_cells = (int64_t)hc.sweep_cells;
    s.tag_cells = (int64_t)hc.tag_cells;
    s.base_cells = (int64_t)hc.base_cells;
    s.levels = levels;
    s.sweep_launches = sweeps;
    s.base_boxes = hc.n_base;
    s.kernel_launches = launches;
    s.retagged_boxes = (int32_t)hc.retag;
    s.resyncs = (int64_t)hc.resyncs;
    s.polls = (int64_t)hc.polls;
    s.sweep_ms = sweep_ms;
    s.device_ms = total_ms;
    return map_device_error(hc.err);
}

// Local alignment (Smith-Waterman) in linear memory, three passes on the node
// grid of the padded sequences (X padded with one sentinel, Y with another, so
// that the corner node never counts as a match):
//   1. a forward KIND_LOCAL sweep with the local floor finds the best score S
//      and the first node e in row-major order that reaches it;
//   2. a sweep of the reversed box (0,0)..e without the floor finds, among the
//      nodes from which a global alignment to e scores S, the largest in
//      row-major order: the start s;
//   3. the edit-kind recursion aligns the substrings between s and e with the
//      scores as costs (match -match, mismatch, gap), canonically; its node path
//      is shifted to the whole grid.
int run_local(Ctx& c, const int32_t* X, int64_t M, const int32_t* Y, int64_t N, int32_t ma, int32_t mm, int32_t g,
              int32_t* path_out, int64_t* K_out, int64_t* score_out, int64_t* se_out) {
    const int64_t Mn = M + 1, Nn = N + 1;
    const int U = sweep_block_cols(KIND_LOCAL, 1), BR = sweep_band_rows(KIND_LOCAL, 1), G = sweep_group_bands(KIND_LOCAL);
    const long long nb_max = (Mn + BR - 1) / BR + 1;
    const size_t fx = align_up((size_t)(M + 2) * 4), fy = align_up((size_t)(N + 2) * 4);
    const Layout L = make_layout(1, Mn, Nn, (long long)(fx + fy), 0);
    const size_t best_off = align_up((size_t)L.total);
    void* wsv = nullptr;
    int rc = workspace(c, best_off + align_up(16 * (size_t)nb_max), &wsv);
    if (rc) return rc;
    char* ws = static_cast<char*>(wsv);
    cudaStream_t st = c.stream;
    const bool xd = is_device_ptr(X), yd = is_device_ptr(Y);
    int32_t* Xp = reinterpret_cast<int32_t*>(ws + L.feat);
    int32_t* Yp = reinterpret_cast<int32_t*>(ws + L.feat + fx);
    cudaError_t e = launch_fill_i32(Xp, M + 2, kEditPad, st);
    if (e == cudaSuccess) e = launch_fill_i32(Yp, N + 2, kEditPad + 1, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(Xp + 1, X, 4 * (size_t)M, xd ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(Yp + 1, Y, 4 * (size_t)N, yd ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    PairDesc pd{};
    pd.X = Xp;
    pd.Y = Yp;
    pd.M = (int32_t)Mn;
    pd.N = (int32_t)Nn;
    pd.esub = mm;
    pd.egap = g;
    pd.ematch = -ma;
    PairDesc* d_pairs = reinterpret_cast<PairDesc*>(ws + L.pairs);
    Box* d_box = reinterpret_cast<Box*>(ws + L.boxA);
    Sweep* d_sweeps = reinterpret_cast<Sweep*>(ws + L.sweeps);
    SweepRes* d_sres = reinterpret_cast<SweepRes*>(ws + L.sres);
    LevelCtl* d_ctl = reinterpret_cast<LevelCtl*>(ws + L.ctl);
    int32_t* d_best = reinterpret_cast<int32_t*>(ws + best_off);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_pairs, &pd, sizeof(pd), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return DTW_ECUDA;

    // one KIND_LOCAL sweep of box (0,0) .. (H-1, W-1): the best node's value and frame cell
    auto pass = [&](int32_t H, int32_t W, int local, int32_t* v, int32_t* p, int32_t* q) -> int {
        Box root{};
        root.pair = 0;
        root.H = H;
        root.W = W;
        root.flags = BOX_ROOT;
        root.known_i = -1;
        root.known_f = NAN;
        LevelCtl ctl0{};
        ctl0.epoch_base = c.epoch;
        cudaError_t err = cudaMemcpyAsync(d_box, &root, sizeof(root), cudaMemcpyHostToDevice, st);
        if (err == cudaSuccess) err = cudaMemcpyAsync(d_ctl, &ctl0, sizeof(ctl0), cudaMemcpyHostToDevice, st);
        if (err == cudaSuccess) err = cudaMemsetAsync(ws + L.bufpool, 0, 8 * (size_t)L.cap_buf, st);
        if (err == cudaSuccess) err = cudaMemsetAsync(d_best, 0, 16 * (size_t)nb_max, st);
        PlanArgs pa{d_box, 1, d_pairs, MODE_COST, KIND_LOCAL, 0, U, BR, G, d_sweeps, d_ctl,
                    L.cap_sweeps, L.cap_buf, L.cap_out, nullptr, 0, false, nullptr};
        pa.local = local;
        pa.tmap = reinterpret_cast<int2*>(ws + L.tmap);
        pa.cap_tickets = L.cap_tickets;
        pa.map_min = c.num_sms;
        if (err == cudaSuccess) err = launch_plan(pa, st);
        LevelCtl hc{};
        if (err == cudaSuccess) err = cudaMemcpyAsync(&hc, d_ctl, sizeof(hc), cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaStreamSynchronize(st);
        if (err != cudaSuccess) return DTW_ECUDA;
        if (hc.err != ERR_NONE) return map_device_error(hc.err);
        c.epoch = hc.epoch_base;
        if (hc.n_bands > nb_max) return DTW_EINTERNAL;
        SweepArgs sa{d_sweeps, d_ctl, reinterpret_cast<unsigned long long*>(ws + L.bufpool), ws + L.outpool, d_sres,
                     1, c.spin_limit, -1};
        sa.best = d_best;
        sa.tmap = reinterpret_cast<const int2*>(ws + L.tmap);
        err = launch_sweep(KIND_LOCAL, 1, false, sa, c.num_sms, hc.n_tickets, st, 0);
        std::vector<int32_t> hb(4 * (size_t)hc.n_bands);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync(hb.data(), d_best, hb.size() * 4, cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaMemcpyAsync(&hc, d_ctl, sizeof(hc), cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaStreamSynchronize(st);
        if (err != cudaSuccess) return DTW_ECUDA;
        if (hc.err != ERR_NONE) return map_device_error(hc.err);
        // bands run down the frame rows: the lexicographic minimum of (value, row, column)
        bool any = false;
        for (long long b = 0; b < hc.n_bands; ++b) {
            const int32_t* r = &hb[4 * b];
            if (!r[3]) return DTW_EINTERNAL;
            if (!any || r[0] < *v || (r[0] == *v && (r[1] < *p || (r[1] == *p && r[2] < *q)))) {
                *v = r[0];
                *p = r[1];
                *q = r[2];
                any = true;
            }
        }
        return any ? DTW_OK : DTW_EINTERNAL;
    };
    int32_t v1 = 0, p1 = 0, q1 = 0;
    rc = pass((int32_t)Mn, (int32_t)Nn, 1, &v1, &p1, &q1);
    if (rc) return rc;
    const int64_t S = -(int64_t)v1;
    *score_out = S;
    for (int k = 0; k < 4; ++k) se_out[k] = 0;
    if (S <= 0) {  // no positive local alignment
        *K_out = 0;
        return DTW_OK;
    }
    const int32_t ae = p1, be = q1;
    int32_t v2 = 0, p2 = 0, q2 = 0;
    rc = pass(ae + 1, be + 1, 2, &v2, &p2, &q2);
    if (rc) return rc;
    // the reversed sweep's values carry the cost of the step out of e: -match or mismatch
    if (v2 + S != -(int64_t)ma && v2 + S != (int64_t)mm) return DTW_EINTERNAL;
    const int32_t as = ae - p2, bs = be - q2;
    if (as < 0 || bs < 0 || as >= ae || bs >= be) return DTW_EINTERNAL;
    // 3. the canonical global alignment of the substrings between s and e
    const int32_t sv[3] = {c.esub, c.egap, c.ematch};
    c.esub = mm;
    c.egap = g;
    c.ematch = -ma;
    const void* xs[1] = {X + as};
    const void* ys[1] = {Y + bs};
    const int64_t ms[1] = {ae - as}, ns[1] = {be - bs};
    int32_t* ps[1] = {path_out};
    int64_t K = 0;
    double cost = 0;
    rc = run_batch(c, 1, xs, ms, ys, ns, 1, KIND_EDIT, true, ps, &K, &cost);
    c.esub = sv[0];
    c.egap = sv[1];
    c.ematch = sv[2];
    if (rc) return rc;
    if (is_device_ptr(path_out)) {
        e = launch_offset_path(path_out, K, as, bs, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return DTW_ECUDA;
    } else {
        for (int64_t t = 0; t < K; ++t) {
            path_out[2 * t] += as;
            path_out[2 * t + 1] += bs;
        }
    }
    *K_out = K;
    se_out[0] = as;
    se_out[1] = bs;
    se_out[2] = ae;
    se_out[3] = be;
    return DTW_OK;
}

int run_plain(Ctx& c, const void* X, int64_t M, const void* Y, int64_t N, int d, int kind, int32_t* path_out,
              int64_t* K_out, double* cost_out) {
    const size_t esize = 4;
    const bool xd = is_device_ptr(X), yd = is_device_ptr(Y), pdv = is_device_ptr(path_out);
    const size_t fx = xd ? 0 : align_up((size_t)M * d * esize), fy = yd ? 0 : align_up((size_t)N * d * esize);
    const size_t fp = pdv ? 0 : align_up(sizeof(int32_t) * 2 * (size_t)(M + N - 1));
    const size_t wb = plain_workspace_bytes(M, N);
    void* wsv = nullptr;
    int rc = workspace(c, fx + fy + fp + wb, &wsv);
    if (rc) return rc;
    char* ws = static_cast<char*>(wsv);
    cudaStream_t st = c.stream;
    cudaError_t e = cudaSuccess;
    PlainProblem pb{X, Y, M, N, d, kind};
    if (!xd) {
        e = cudaMemcpyAsync(ws, X, (size_t)M * d * esize, cudaMemcpyHostToDevice, st);
        pb.X = ws;
    }
    if (e == cudaSuccess && !yd) {
        e = cudaMemcpyAsync(ws + fx, Y, (size_t)N * d * esize, cudaMemcpyHostToDevice, st);
        pb.Y = ws + fx;
    }
    if (e != cudaSuccess) return DTW_ECUDA;
    int32_t* dpath = pdv ? path_out : reinterpret_cast<int32_t*>(ws + fx + fy);
    Timer T{c.timing != 0, st, {}};
    cudaEvent_t t0 = c.timing ? T.mark() : nullptr;
    long long cells = 0;
    rc = plain_align(pb, dpath, cost_out, K_out, ws + fx + fy + fp, wb, st, &cells);
    if (rc) return rc;
    if (!pdv) {
        e = cudaMemcpyAsync(path_out, dpath, sizeof(int32_t) * 2 * (size_t)*K_out, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return DTW_ECUDA;
    }
    dtw_stats& s = c.stats;
    s = dtw_stats{};
    s.problem_cells = M * N;
    s.sweep_cells = cells;
    if (c.timing) {
        cudaEvent_t t1 = T.mark();
        cudaEventSynchronize(t1);
        s.device_ms = elapsed(t0, t1);
    }
    return DTW_OK;
}

}  // namespace

namespace dtwb {
namespace {
std::atomic<int> g_split_windows{kSplitWindowsDefault};
}
int split_windows_option() { return g_split_windows.load(std::memory_order_relaxed); }
void set_split_windows_option(int windows) { g_split_windows.store(windows, std::memory_order_relaxed); }
}  // namespace dtwb

// ================================================================= C ABI

extern "C" {

int64_t dtw_align(const void* X, int64_t M, const void* Y, int64_t N, int32_t d, int32_t cost_kind,
                  int32_t* path_out, double* cost_out) {
    int kind;
    bool plain;
    int rc = check_kind(cost_kind, d, &kind, &plain);
    if (rc) return rc;
    if (!X || !Y || !path_out || !cost_out || M < 1 || N < 1) return DTW_EINVAL;
    Ctx& c = ctx();
    std::lock_guard<std::mutex> g(c.mu);
    rc = ensure_device(c);
    if (rc) return rc;
    int64_t K = 0;
    if (plain) {
        rc = run_plain(c, X, M, Y, N, d, kind, path_out, &K, cost_out);
    } else {
        const void* xs[1] = {X};
        const void* ys[1] = {Y};
        int32_t* ps[1] = {path_out};
        rc = run_batch(c, 1, xs, &M, ys, &N, d, kind, true, ps, &K, cost_out);
    }
    return rc ? rc : K;
}

int dtw_cost(const void* X, int64_t M, const void* Y, int64_t N, int32_t d, int32_t cost_kind, double* cost_out) {
    int kind;
    bool plain;
    int rc = check_kind(cost_kind, d, &kind, &plain);
    if (rc) return rc;
    if (plain || !X || !Y || !cost_out || M < 1 || N < 1) return DTW_EINVAL;
    Ctx& c = ctx();
    std::lock_guard<std::mutex> g(c.mu);
    rc = ensure_device(c);
    if (rc) return rc;
    const void* xs[1] = {X};
    const void* ys[1] = {Y};
    return run_batch(c, 1, xs, &M, ys, &N, d, kind, false, nullptr, nullptr, cost_out);
}

int dtw_align_batch(int32_t B, const void* const* X, const int64_t* M, const void* const* Y, const int64_t* N,
                    int32_t d, int32_t cost_kind, int32_t* const* path_out, int64_t* K_out, double* cost_out) {
    int kind;
    bool plain;
    int rc = check_kind(cost_kind, d, &kind, &plain);
    if (rc) return rc;
    if (B < 1 || !X || !M || !Y || !N || !path_out || !K_out || !cost_out || plain) return DTW_EINVAL;
    Ctx& c = ctx();
    std::lock_guard<std::mutex> g(c.mu);
    rc = ensure_device(c);
    if (rc) return rc;
    return run_batch(c, B, X, M, Y, N, d, kind, true, path_out, K_out, cost_out);
}

int dtw_set_stream(void* cuda_stream) {
    Ctx& c = ctx();
    std::lock_guard<std::mutex> g(c.mu);
    c.stream = static_cast<cudaStream_t>(cuda_stream);
    return DTW_OK;
}

int dtw_set_budget(uint64_t bytes) {
    Ctx& c = ctx();
    std::lock_guard<std::mutex> g(c.mu);
    c.budget = bytes;
    serve_set_budget(bytes);
    return DTW_OK;
}

int dtw_set_arena(void* device_ptr, uint64_t bytes) {
    Ctx& c = ctx();
    std::lock_guard<std::mutex> g(c.mu);
    if (device_ptr && (reinterpret_cast<uintptr_t>(device_ptr) & 255)) return DTW_EINVAL;
    c.arena = device_ptr;
    c.arena_bytes = device_ptr ? bytes : 0;
    // boundary words must not carry a future epoch by accident
    if (device_ptr && cudaMemsetAsync(device_ptr, 0, bytes, c.stream) != cudaSuccess) return DTW_ECUDA;
    return DTW_OK;
}

size_t dtw_footprint(int64_t M, int64_t N, int32_t d, int32_t cost_kind) {
    if (M < 1 || N < 1 || d < 1) return 0;
    const int windows = split_windows_option();
    if (cost_kind & DTW_PLAIN_F64) {
        return align_up((size_t)(M + N) * d * 4) + 3 * 256 + align_up(8 * (size_t)(M + N)) +
               plain_workspace_bytes(M, N);
    }
    if ((cost_kind & 0xff) == DTW_EDIT_I32) {  // the node grid over the padded sequences
        const Layout L = make_layout(1, M + 1, N + 1,
                                     (long long)align_up((size_t)(M + 2) * 4) + (long long)align_up((size_t)(N + 2) * 4),
                                     M + N + 1, windows, split_win_rows(KIND_EDIT));
        return L.total;
    }
    const int kind = (cost_kind & 0xff) == DTW_ABS_I32 ? KIND_ABS : KIND_EUC;
    const Layout L = make_layout(1, M, N, (long long)align_up((size_t)M * d * 4) + (long long)align_up((size_t)N * d * 4),
                                 M + N - 1, windows, split_win_rows(kind));
    return L.total;
}

int dtw_local_align(const int32_t* X, int64_t M, const int32_t* Y, int64_t N, int32_t match, int32_t mismatch,
                    int32_t gap, int32_t* path_out, int64_t* K_out, int64_t* score_out, int64_t* se_out) {
    if (!X || !Y || !path_out || !K_out || !score_out || !se_out || M < 1 || N < 1 || M >= (1LL << 30) ||
        N >= (1LL << 30))
        return DTW_EINVAL;
    if (match < 0 || mismatch < 0 || gap < 0 || match > (1 << 20) || mismatch > (1 << 20) || gap > (1 << 20))
        return DTW_EINVAL;
    if ((M + N + 2) * (long long)std::max(match, std::max(mismatch, gap)) >= (1LL << 29)) return DTW_EOVERFLOW;
    Ctx& c = ctx();
    std::lock_guard<std::mutex> g(c.mu);
    int rc = ensure_device(c);
    if (rc) return rc;
    return run_local(c, X, M, Y, N, match, mismatch, gap, path_out, K_out, score_out, se_out);
}

int dtw_path_discrepancy(const int32_t* P1, int64_t K1, const int32_t* P2, int64_t K2, int64_t M, int64_t N,
                         int32_t* err_out, int32_t* max_out) {
    if (!P1 || !P2 || !err_out || M < 1 || N < 1) return DTW_EINVAL;
    const int64_t kmin = M > N ? M : N, kmax = M + N - 1;
    if (K1 < kmin || K1 > kmax || K2 < kmin || K2 > kmax) return DTW_EINVAL;
    Ctx& c = ctx();
    std::lock_guard<std::mutex> g(c.mu);
    int rc = ensure_device(c);
    if (rc) return rc;
    const bool d1 = is_device_ptr(P1), d2 = is_device_ptr(P2), de = is_device_ptr(err_out);
    const size_t b1 = sizeof(int32_t) * 2 * (size_t)K1, b2 = sizeof(int32_t) * 2 * (size_t)K2;
    const size_t s1 = d1 ? 0 : align_up(b1), s2 = d2 ? 0 : align_up(b2), se = de ? 0 : align_up(b1);
    const size_t used = s1 + s2 + se + discrepancy_workspace_bytes(M, N);
    void* wsv = nullptr;
    rc = workspace(c, used, &wsv);
    if (rc) return rc;
    char* ws = static_cast<char*>(wsv);
    cudaStream_t st = c.stream;
    const int32_t* p1 = d1 ? P1 : reinterpret_cast<const int32_t*>(ws);
    const int32_t* p2 = d2 ? P2 : reinterpret_cast<const int32_t*>(ws + s1);
    int32_t* err = de ? err_out : reinterpret_cast<int32_t*>(ws + s1 + s2);
    cudaError_t e = cudaSuccess;
    if (!d1) e = cudaMemcpyAsync(ws, P1, b1, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !d2) e = cudaMemcpyAsync(ws + s1, P2, b2, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return DTW_ECUDA;
    rc = path_discrepancy(p1, K1, p2, K2, M, N, err, max_out, ws + s1 + s2 + se, c.num_sms, st);
    if (rc == DTW_OK && !de) {
        e = cudaMemcpyAsync(err_out, err, b1, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = DTW_ECUDA;
    }
    // the workspace also holds epoch-stamped boundary words of later alignments:
    // leave no stray value behind that could carry a future epoch
    if (cudaMemsetAsync(ws, 0, used, st) != cudaSuccess && rc == DTW_OK) rc = DTW_ECUDA;
    return rc;
}

const char* dtw_strerror(int status) {
    switch (status) {
        case DTW_OK: return "ok";
        case DTW_PENDING: return "pending";
        case DTW_EINVAL: return "invalid argument";
        case DTW_ENOMEM: return "out of device memory or over budget";
        case DTW_ECUDA: return "CUDA runtime error";
        case DTW_ETIMEOUT: return "device-side wait timed out";
        case DTW_EOVERFLOW: return "integer accumulator range exceeded";
        case DTW_EBUSY: return "queue full";
        case DTW_EINTERNAL: return "internal consistency check failed";
        default: return "unknown status";
    }
}

int dtw_get_stats(dtw_stats* out) {
    if (!out) return DTW_EINVAL;
    Ctx& c = ctx();
    std::lock_guard<std::mutex> g(c.mu);
    *out = c.stats;
    return DTW_OK;
}

int dtw_set_option(int32_t key, int64_t value) {
    Ctx& c = ctx();
    std::lock_guard<std::mutex> g(c.mu);
    switch (key) {
        case DTW_OPT_TIMING: c.timing = value != 0; return DTW_OK;
        case DTW_OPT_BASE_AREA:
            if (value < 4 || value > kBaseAreaMax) return DTW_EINVAL;
            c.base_area = value;
            return DTW_OK;
        case DTW_OPT_SPIN_LIMIT:
            if (value < 1 || value > (1LL << 30)) return DTW_EINVAL;
            c.spin_limit = (int)value;
            return DTW_OK;
        case DTW_OPT_SKIP_PUBLISH: c.skip_publish = value; return DTW_OK;
        case DTW_OPT_GRAPH: c.use_graph = value != 0; return DTW_OK;
        case DTW_OPT_SWEEP_VARIANT:
            if (value < 0 || value >= kSweepVariants) return DTW_EINVAL;
            c.variant = (int)value;
            return DTW_OK;
        case DTW_OPT_EDIT_SUB:
            if (value < 0 || value > (1 << 20)) return DTW_EINVAL;
            c.esub = (int32_t)value;
            return DTW_OK;
        case DTW_OPT_EDIT_GAP:
            if (value < 0 || value > (1 << 20)) return DTW_EINVAL;
            c.egap = (int32_t)value;
            return DTW_OK;
        case DTW_OPT_FUSED_SPLIT:
            if (value < 0 || value > 2) return DTW_EINVAL;
            c.fused_split = (int)value;
            return DTW_OK;
        case DTW_OPT_SPLIT_WINDOWS:
            if (value < 1 || value > kSplitWinMax) return DTW_EINVAL;
            c.split_windows = (int)value;
            set_split_windows_option((int)value);
            return DTW_OK;
        case DTW_OPT_NOALLOC_EPOCH:
            if (value < 0 || value > 0xFFFFFFFFLL) return DTW_EINVAL;
            noalloc_set_epoch(value);
            return DTW_OK;
        default: return DTW_EINVAL;
    }
}

}  // extern "C"
