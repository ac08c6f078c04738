// Per-level kernels of the divide-and-conquer recursion (Section 3.2,
// Algorithm 2): planning the sweeps of every box of a level, choosing each box's
// pivot on its split row (Lemmas 1 and 2), emitting the two child boxes that
// share the pivot, finishing small boxes with a full-table DP and backtrace
// (Section 2.1), and assembling the per-pair warping paths.
#include <climits>
#include <type_traits>

#include "dtw_common.cuh"
#include "dtw_kernels.h"
#include "split.cuh"

namespace dtwb {

// ---------------------------------------------------------------- block scan

// Exclusive scan of one long long per thread over a 1024-thread block.
__device__ long long block_excl_scan(long long v, long long* total) {
    __shared__ long long warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        long long w = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    long long base = wid ? warp_sums[wid - 1] : 0;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return base + x - v;
}

// Four exclusive scans at once (one long long of each per thread), with the
// barriers of one.
__device__ void block_excl_scan4(const long long (&v)[4], long long (&e)[4], long long (&total)[4]) {
    __shared__ long long warp_sums4[32][4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long x[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = v[k];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long y = __shfl_up_sync(kFull, x[k], o);
            if (lane >= o) x[k] += y;
        }
    }
    if (lane == 31) {
#pragma unroll
        for (int k = 0; k < 4; ++k) warp_sums4[wid][k] = x[k];
    }
    __syncthreads();
    if (wid == 0) {
        long long w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = lane < nw ? warp_sums4[lane][k] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const long long y = __shfl_up_sync(kFull, w[k], o);
                if (lane >= o) w[k] += y;
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) warp_sums4[lane][k] = w[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        e[k] = (wid ? warp_sums4[wid - 1][k] : 0) + x[k] - v[k];
        total[k] = warp_sums4[nw - 1][k];
    }
    __syncthreads();
}

// ---------------------------------------------------------------- plan

// Largest band-group count per sweep the ticket map handles (one bucket per
// plan thread); longer sweeps use the plain ticket order.
constexpr int kTmapBuckets = 1024;

// One block of 1024 threads.  Every box owns two sweep slots.  An aligned box
// gets a forward half sweep (frame rows 0..r+h) and a backward half sweep
// (rows r-h..P-1 of the reversed box), both ending on the window of split rows
// r-h..r+h; a box flagged BOX_TAG gets one tagged forward sweep of the whole box
// (second slot empty); in cost mode the single slot sweeps the whole box.
// Then band tickets, pool offsets, epochs and the level counters.
__global__ void __launch_bounds__(1024) plan_kernel(PlanArgs a) {
    __shared__ long long carry[4];
    __shared__ unsigned long long cells_sh[2];
    __shared__ int ntag_sh;
    __shared__ uint32_t ep_base;
    const int nslot = a.mode == MODE_COST ? 1 : 2;
    if (threadIdx.x < 4) carry[threadIdx.x] = 0;
    if (threadIdx.x < 2) cells_sh[threadIdx.x] = 0;
    if (threadIdx.x == 0) ntag_sh = 0;
    __shared__ int nbox_sh;
    if (threadIdx.x == 0) {
        ep_base = a.ctl->epoch_base;
        nbox_sh = a.n_boxes >= 0 ? a.n_boxes : a.ctl->n_next;
    }
    __syncthreads();
    const int n_boxes = nbox_sh;
    unsigned long long my_cells = 0, my_tag = 0;
    const int nsw = n_boxes * nslot;
    for (int base = 0; base < nsw; base += blockDim.x) {
        const int s = base + threadIdx.x;
        const bool valid = s < nsw;
        Sweep sw = {};
        long long nb = 0, nbuf = 0, nout = 0, nit = 0;
        int wbands = 0;  // bands holding split rows (the fused split waits for them)
        if (valid) {
            const int bi = s / nslot, dir = s % nslot;
            const Box b = a.boxes[bi];
            if (a.copy_to && dir == 0) a.copy_to[bi] = b;
            const PairDesc pd = a.pairs[b.pair];
            Geom g = geom_of(b);
            if (a.local) {  // local sweeps keep frame rows along X (row-major order of the best node)
                g.axis = 0;
                g.P = b.H;
                g.Q = b.W;
                g.r = (g.P - 1) / 2;
            }
            sw.box = bi;
            sw.dir = dir;
            sw.axis = g.axis;
            sw.Q = g.Q;
            sw.tag_row = -1;
            sw.nout = 0;
            sw.out_row0 = 0;
            sw.onw = 0;
            sw.owin = 1;
            sw.ospace = 1;
            if (a.mode == MODE_COST) {
                sw.rows = g.P;
            } else if (b.flags & BOX_TAG) {
                if (dir == 0) atomicAdd(&ntag_sh, 1);
                sw.rows = dir == 0 ? g.P : 0;
                sw.out_row0 = g.r;
                sw.nout = dir == 0 ? 1 : 0;
                sw.onw = sw.nout;
                sw.tag_row = g.r;
                wbands = sw.nout;
            } else {
                // the windows stay inside rows 1..P-2, so every child is strictly
                // shorter than the box along the cut side
                const int h = max(0, min(a.halo, min(g.r - 1, g.P - 2 - g.r)));
                const int ow = 2 * h + 1;
                // nw windows of split rows centred on r + (t - c) S, t = 0..nw-1,
                // c = (nw-1)/2, S = P/(nw+1): the middle one on row r, the
                // children nw+1 pieces of about P/(nw+1) rows.  The forward sweep
                // runs to the last window, the backward one to the first.
                int nw = 1, S = ow, r0 = g.r, rl = g.r;
                for (int cand = (min(a.nwin, kSplitWinMax) - 1) | 1; cand > 1; cand -= 2) {
                    const int cs = g.P / (cand + 1), cc = (cand - 1) / 2;
                    const int c0 = g.r - cc * cs, cl = g.r + (cand - 1 - cc) * cs;
                    if (cand * ow <= kOutRowsMax && cs - ow >= kWinGap && c0 - h >= 1 && cl + h <= g.P - 2) {
                        nw = cand;
                        S = cs;
                        r0 = c0;
                        rl = cl;
                        break;
                    }
                }
                sw.rows = dir == 0 ? rl + h + 1 : g.P - r0 + h;
                sw.onw = nw;
                sw.owin = ow;
                sw.ospace = S;
                sw.nout = nw * ow;
                // both sweeps end on their last window (rows r_t-h..r_t+h of every
                // window, in each sweep's own frame order)
                sw.out_row0 = dir == 0 ? r0 - h : g.P - 1 - (rl + h);
                for (int t = 0, last = -1; t < nw; ++t) {
                    const int w0 = sw.out_row0 + t * S;
                    for (int bb = max(w0 / a.BR, last + 1); bb <= (w0 + ow - 1) / a.BR; ++bb) {
                        ++wbands;
                        last = bb;
                    }
                }
            }
            sw.nblk = sw.rows > 0 ? (g.Q + a.U - 1) / a.U : 0;
            sw.ostride = sw.nblk * a.U;
            sw.nbands = sw.rows > 0 ? (sw.rows + a.BR - 1) / a.BR : 0;
            sw.rowseq = g.axis ? pd.Y : pd.X;
            sw.colseq = g.axis ? pd.X : pd.Y;
            const int rb0 = g.axis ? b.j0 : b.i0, rlen = g.axis ? b.W : b.H;
            const int cb0 = g.axis ? b.i0 : b.j0, clen = g.axis ? b.H : b.W;
            if (dir == 0 && a.local != 2) {
                sw.rbase = rb0;
                sw.rstep = 1;
                sw.cbase = cb0;
                sw.cstep = 1;
            } else {  // the reversed series X_R, Y_R of Algorithm 2
                // edit distance: the step into reversed node p consumes forward symbol p + 1
                const int shift = edit_kind(a.kind) ? 1 : 0;
                sw.rbase = rb0 + rlen - 1 + shift;
                sw.rstep = -1;
                sw.cbase = cb0 + clen - 1 + shift;
                sw.cstep = -1;
            }
            sw.esub = pd.esub;
            sw.egap = pd.egap;
            sw.ematch = pd.ematch;
            sw.floor = a.local == 1 ? 1 : 0;
            nb = sw.nbands;
            // a block that must take a group of G bands of one sweep (the BF16
            // form: the M rows of its MMAs; the d = 64 FP32-cost kinds: their
            // tight frame ring): in the plain ticket order each sweep's bands
            // start on a whole group (the padding bands stay idle)
            if (a.whole_groups) nb = (nb + a.G - 1) / a.G * a.G;
            // boundary words per column: one for an untagged integer sweep, two otherwise
            const int nw = (int_kind(a.kind) && sw.tag_row < 0) ? 1 : 2;
            nbuf = (long long)nw * sw.nblk * a.U;
            nout = (long long)sw.nout * sw.ostride;
            // split work: the forward slot of an aligned box owns the box's column chunks
            if (a.mode != MODE_COST && dir == 0) {
                const int ic = split_item_cols(sw.onw);
                nit = (b.flags & BOX_TAG) ? 1 : (long long)sw.onw * ((g.Q + ic - 1) / ic);
                if (a.box_done) a.box_done[bi] = 0;
            }
            sw.nitems = (int)nit;
            my_cells += (unsigned long long)sw.rows * (unsigned long long)g.Q;
            if (sw.tag_row >= 0) my_tag += (unsigned long long)(sw.rows - sw.tag_row) * g.Q;
        }
        const long long v4[4] = {nb, nbuf, nout, nit};
        long long e4[4], t4[4];
        block_excl_scan4(v4, e4, t4);  // ends with a barrier: carry[] is read by all
        if (valid) {
            sw.band_begin = carry[0] + e4[0];
            sw.epoch0 = ep_base + (uint32_t)(carry[0] + e4[0]);
            sw.buf_off = carry[1] + e4[1];
            sw.out_off = carry[2] + e4[2];
            sw.item0 = (int)(carry[3] + e4[3]);
            if (s < a.cap_sweeps) {
                a.sweeps[s] = sw;
                if (a.prog) {
                    // split-row progress: bands holding split rows that have ended, of wbands
                    int* pw = a.prog + (size_t)s * kProgWords;
                    pw[0] = 0;
                    pw[1] = wbands;
                    pw[2] = 0;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x < 4) carry[threadIdx.x] += t4[threadIdx.x];
        __syncthreads();
    }
    // warp sums first: one shared atomic per warp instead of per thread
    for (int o = 16; o; o >>= 1) {
        my_cells += __shfl_down_sync(kFull, my_cells, o);
        my_tag += __shfl_down_sync(kFull, my_tag, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&cells_sh[0], my_cells);
        atomicAdd(&cells_sh[1], my_tag);
    }
    __syncthreads();
    // Ticket map, group-major: ticket t -> (sweep, band group j), every sweep's
    // first group of G bands first, then every sweep's second group, and so on
    // (sweeps with more groups first within a round).  A block then takes a
    // group whose band above started about one round earlier, instead of a
    // group far down a sweep whose first band has only just started.
    __shared__ int tm_hist[kTmapBuckets];  // sweeps per group count; later per-bucket fill counters
    __shared__ int tm_cnt[kTmapBuckets];   // tm_cnt[j]: sweeps with more than j groups
    __shared__ int tm_off[kTmapBuckets];   // first ticket of round j
    __shared__ int tm_ok;
    __shared__ long long tm_total;
    bool map_on = false;
    if (a.tmap != nullptr && (long long)nsw <= a.cap_sweeps && (carry[0] + a.G - 1) / a.G > a.map_min) {
        for (int i = threadIdx.x; i < kTmapBuckets; i += blockDim.x) tm_hist[i] = 0;
        if (threadIdx.x == 0) tm_ok = 1;
        __syncthreads();
        // deep levels hold thousands of sweeps with the same few group counts:
        // the lanes of a warp with equal counts share one shared-memory atomic
        for (int base = 0; base < nsw; base += blockDim.x) {
            const int s = base + threadIdx.x;
            int ng = s < nsw ? (a.sweeps[s].nbands + a.G - 1) / a.G : 0;
            if (ng >= kTmapBuckets) {
                tm_ok = 0;
                ng = 0;
            }
            const unsigned peers = __match_any_sync(kFull, ng);
            if (ng > 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&tm_hist[ng], __popc(peers));
        }
        __syncthreads();
        if (tm_ok) {
            long long tot;
            // suffix sums of the histogram: a scan of it reversed (one bucket per thread)
            const int r = threadIdx.x;
            const long long e = block_excl_scan(tm_hist[kTmapBuckets - 1 - r], &tot);
            tm_cnt[kTmapBuckets - 1 - r] = (int)e;
            __syncthreads();
            const long long o = block_excl_scan(tm_cnt[threadIdx.x], &tot);
            tm_off[threadIdx.x] = (int)o;
            tm_hist[threadIdx.x] = 0;
            if (threadIdx.x == 0) {
                tm_total = tot;
                if (tot > a.cap_tickets) tm_ok = 0;
            }
            __syncthreads();
            if (tm_ok) {
                const int lane = threadIdx.x & 31;
                for (int base = 0; base < nsw; base += blockDim.x) {
                    const int s = base + threadIdx.x;
                    const int ng = s < nsw ? (a.sweeps[s].nbands + a.G - 1) / a.G : 0;
                    // descending group count: bucket ng starts after every sweep with
                    // more groups; lanes with equal counts take consecutive places
                    const unsigned peers = __match_any_sync(kFull, ng);
                    const int leader = __ffs(peers) - 1;
                    int first = 0;
                    if (ng > 0 && lane == leader) first = atomicAdd(&tm_hist[ng], __popc(peers));
                    first = __shfl_sync(kFull, first, leader);
                    if (ng > 0) {
                        const int pos = tm_cnt[ng] + first + __popc(peers & ((1u << lane) - 1u));
                        for (int j = 0; j < ng; ++j) a.tmap[tm_off[j] + pos] = make_int2(s, j);
                    }
                }
            }
        }
        __syncthreads();
        map_on = tm_ok != 0;
    }
    if (threadIdx.x == 0) {
        const long long total_bands = carry[0];
        const bool fits = (long long)nsw <= a.cap_sweeps && carry[1] <= a.cap_buf && carry[2] <= a.cap_out &&
                          (a.mode == MODE_COST || carry[3] <= a.cap_items);
        LevelCtl* c = a.ctl;
        c->ticket = 0;
        c->split_ticket = 0;
        c->n_next = 0;
        c->n_cur = n_boxes;
        c->n_tag = ntag_sh;
        if (a.reset_base) c->n_base = 0;
        c->need_buf = carry[1];
        c->epoch_base = ep_base + (uint32_t)total_bands + 1u;
        if (fits) {
            c->n_sweeps = nsw;
            c->n_items = (int)carry[3];
            c->n_bands = total_bands;
            c->n_tickets = map_on ? tm_total : (total_bands + a.G - 1) / a.G;
            c->tmap_on = map_on ? 1 : 0;
            c->sweep_cells += cells_sh[0];
            c->tag_cells += cells_sh[1];
        } else {
            c->n_sweeps = 0;
            c->n_items = 0;
            c->n_bands = 0;
            c->n_tickets = 0;
            c->tmap_on = 0;
            set_error(c, ERR_CAPACITY, 0);
        }
    }
}

cudaError_t launch_plan(const PlanArgs& a, cudaStream_t st) {
    plan_kernel<<<1, 1024, 0, st>>>(a);
    return cudaGetLastError();
}

// Work items of a level: every column chunk of every box's split rows (one
// item for a tagged box).  Each item writes its partial minima; the item that
// finishes a box last (per-box counter) merges them and emits the children.
// Two blocks per SM for the integer kinds (their item work fits in 128 registers).
template <int KIND, int DIM>
__global__ void __launch_bounds__(256, int_kind(KIND) ? 2 : 1) split_kernel(SplitArgs a) {
    // after a planning or sweep error the sweep outputs are not valid
    if (ld_relaxed(&a.ctl->err) != ERR_NONE) return;
    const int n_items = a.n_items >= 0 ? a.n_items : a.ctl->n_items;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) split_item<KIND, DIM>(a, it, nullptr);
}

cudaError_t launch_split(const SplitArgs& a, cudaStream_t st) {
    const int cap = 8 * (a.num_sms > 0 ? a.num_sms : 148);
    int grid = cap;  // counts read on the device: a full grid
    if (a.n_items >= 0 && a.n_boxes >= 0) {
        if (a.n_boxes == 0 || a.n_items == 0) return cudaSuccess;
        if (a.n_items < grid) grid = a.n_items;
    }
    if (a.kind == KIND_ABS) split_kernel<KIND_ABS, 1><<<grid, 256, 0, st>>>(a);
    else if (a.kind == KIND_EDIT) split_kernel<KIND_EDIT, 1><<<grid, 256, 0, st>>>(a);
    else if (a.kind == KIND_EUCB) split_kernel<KIND_EUCB, 64><<<grid, 256, 0, st>>>(a);
    else if (a.kind == KIND_EUCF && a.d == 12) split_kernel<KIND_EUCF, 12><<<grid, 256, 0, st>>>(a);
    else if (a.kind == KIND_EUCF && a.d == 64) split_kernel<KIND_EUCF, 64><<<grid, 256, 0, st>>>(a);
    else if (a.kind == KIND_EUCF) split_kernel<KIND_EUCF, 0><<<grid, 256, 0, st>>>(a);
    else if (a.d == 12) split_kernel<KIND_EUC, 12><<<grid, 256, 0, st>>>(a);
    else if (a.d == 64) split_kernel<KIND_EUC, 64><<<grid, 256, 0, st>>>(a);
    else split_kernel<KIND_EUC, 0><<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}


// ---------------------------------------------------------------- base case

// Shared memory per warp: 2-bit backpointers of up to kBaseAreaMax cells
// (rows are the shorter side, 16 pointers per word, each row word-aligned) and
// the boundary row between consecutive 32-row bands.
constexpr long long isqrt_ceil(long long a) {
    long long r = 0;
    while (r * r < a) ++r;
    return r;
}
constexpr int kPtrWords = (int)(kBaseAreaMax / 16 + isqrt_ceil(kBaseAreaMax)) + 1;  // P*ceil(Q/16) <= A/16 + sqrt(A)
constexpr int kRowBuf = (int)(kBaseAreaMax / 32);          // Q < A/32 whenever P > 32
constexpr int kBaseWarps = 2;

template <int KIND>
struct BaseSmem {
    uint32_t ptr[kBaseWarps][kPtrWords];
    typename AccOf<KIND>::T row[kBaseWarps][kRowBuf];
};

// One warp per box: full-table DP with backpointers (first minimum in the order
// DIAG, UP, LEFT; Section 2.1), then a backtrace from the box's last cell that
// records, per global row, the range of path columns.
template <int KIND, int DIM>
__global__ void __launch_bounds__(32 * kBaseWarps) base_kernel(BaseArgs a) {
    using Acc = typename AccOf<KIND>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BaseSmem<KIND>& sm = *reinterpret_cast<BaseSmem<KIND>*>(smem_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const Acc INF = AccOf<KIND>::inf();
    const int n_base = a.n_base >= 0 ? a.n_base : a.ctl->n_base;
    for (int bi = blockIdx.x * kBaseWarps + w; bi < n_base; bi += gridDim.x * kBaseWarps) {
        const Box b = a.base[bi];
        const PairDesc pd = a.pairs[b.pair];
        // frame: rows along the shorter side
        const int axis = b.H <= b.W ? 0 : 1;
        const int P = axis ? b.W : b.H, Q = axis ? b.H : b.W;
        const bool vf = axis == 0;  // vertical frame move is UP
        const int QW = (Q + 15) >> 4;
        const void* rs = axis ? pd.Y : pd.X;
        const void* cs = axis ? pd.X : pd.Y;
        const int rbase = axis ? b.j0 : b.i0, cbase = axis ? b.i0 : b.j0;
        uint32_t* ptr = sm.ptr[w];
        Acc* row = sm.row[w];
        Acc end_v = INF;
        for (int band = 0; band * 32 < P; ++band) {
            const int p = band * 32 + lane;
            const bool rowok = p < P;
            Frame<KIND, DIM> xr;
            xr.load(rs, rbase + (rowok ? p : P - 1), a.d);
            Acc left = INF, cur = INF;
            Acc dprev = (p == 0) ? AccOf<KIND>::zero() : INF;  // D(p-1, q-1)
            uint32_t word = 0;
            for (int s = 0; s < Q + 31; ++s) {
                const int q = s - lane;
                Acc up = shfl_up1(cur);
                const bool act = rowok && q >= 0 && q < Q;
                if (lane == 0) up = (band == 0 || !act) ? INF : row[q];
                if (act) {
                    Frame<KIND, DIM> yc;
                    yc.load(cs, cbase + q, a.d);
                    // edit distance: delta on the diagonal move, the gap on every move
                    const auto c = [&]() {
                        if constexpr (edit_kind(KIND)) return pd.egap;
                        else return frame_cost(xr, yc);
                    }();
                    const Acc dd = [&]() {
                        if constexpr (edit_kind(KIND))
                            return dprev + edit_delta(xr.v, yc.v, pd.ematch, pd.esub, pd.egap);
                        else return dprev;
                    }();
                    const Acc m = min3(dd, up, left);
                    uint32_t pt;
                    if (p == 0 && q == 0) pt = 3;
                    else if (dd == m) pt = 0;
                    else if (vf) pt = (up == m) ? 1 : 2;
                    else pt = (left == m) ? 2 : 1;
                    if constexpr (KIND == KIND_ABS) cur = (Acc)__sad(xr.v, yc.v, (unsigned)m);  // |x - y| + m
                    else cur = m + c;
                    left = cur;
                    dprev = up;
                    word |= pt << (2 * (q & 15));
                    if ((q & 15) == 15 || q == Q - 1) {
                        ptr[p * QW + (q >> 4)] = word;
                        word = 0;
                    }
                    if (lane == 31 && band * 32 + 32 < P) row[q] = cur;
                    if (p == P - 1 && q == Q - 1) end_v = cur;
                }
            }
            __syncwarp();
        }
        // the box cost and its consistency with the parent's split
        for (int o = 16; o; o >>= 1) {
            const Acc t = shfl_down(end_v, o);
            end_v = acc_min(end_v, t);
        }
        if (lane == 0) {
            if constexpr (int_kind(KIND)) {
                if (b.known_i >= 0 && b.known_i != (long long)end_v) set_error(a.ctl, ERR_CONSIST, 20);
                if (b.flags & BOX_ROOT) a.pres[b.pair].cost_i = end_v;
            } else {
                if (b.flags & BOX_ROOT) a.pres[b.pair].cost_f = to_double(end_v);
            }
            atomicAdd(&a.ctl->base_cells, (unsigned long long)P * (unsigned long long)Q);
            // backtrace: per global row, the range of path columns
            int p = P - 1, q = Q - 1;
            int32_t* jlo = a.jlo + pd.row_off;
            int32_t* jhi = a.jhi + pd.row_off;
            for (int guard = 0; guard < P + Q; ++guard) {
                const int i = axis ? b.i0 + q : b.i0 + p;
                const int j = axis ? b.j0 + p : b.j0 + q;
                atomicMin(jlo + i, j);
                atomicMax(jhi + i, j);
                const uint32_t pt = (ptr[p * QW + (q >> 4)] >> (2 * (q & 15))) & 3u;
                if (pt == 3) break;
                if (pt == 0) {
                    --p;
                    --q;
                } else if (pt == 1) {
                    --p;
                } else {
                    --q;
                }
                if (p < 0 || q < 0) {
                    set_error(a.ctl, ERR_PATH, 21);
                    break;
                }
            }
        }
        __syncwarp();
    }
}

template <int KIND, int DIM>
static cudaError_t launch_base_t(const BaseArgs& a, cudaStream_t st) {
    const size_t smem = sizeof(BaseSmem<KIND>);
    cudaError_t e = cudaFuncSetAttribute(base_kernel<KIND, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int grid = a.n_base >= 0 ? (a.n_base + kBaseWarps - 1) / kBaseWarps : 1184;
    if (grid > 65535) grid = 65535;
    base_kernel<KIND, DIM><<<grid, 32 * kBaseWarps, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_base(const BaseArgs& a, cudaStream_t st) {
    if (a.n_base == 0) return cudaSuccess;
    if (a.kind == KIND_ABS) return launch_base_t<KIND_ABS, 1>(a, st);
    if (a.kind == KIND_EDIT) return launch_base_t<KIND_EDIT, 1>(a, st);
    if (a.kind == KIND_EUCB) return launch_base_t<KIND_EUCB, 64>(a, st);
    if (a.kind == KIND_EUCF) {
        if (a.d == 12) return launch_base_t<KIND_EUCF, 12>(a, st);
        if (a.d == 64) return launch_base_t<KIND_EUCF, 64>(a, st);
        return launch_base_t<KIND_EUCF, 0>(a, st);
    }
    if (a.d == 12) return launch_base_t<KIND_EUC, 12>(a, st);
    if (a.d == 64) return launch_base_t<KIND_EUC, 64>(a, st);
    return launch_base_t<KIND_EUC, 0>(a, st);
}

// ---------------------------------------------------------------- path assembly

// One block per pair: lengths of the per-row column runs, their exclusive scan
// (the row offsets in the path) and the structural checks of a warping path.
__global__ void __launch_bounds__(1024) assemble_scan_kernel(AssembleArgs a) {
    const int pb = a.idx ? a.idx[blockIdx.x] : blockIdx.x;
    const PairDesc pd = a.pairs[pb];
    const int32_t* jlo = a.jlo + pd.row_off;
    const int32_t* jhi = a.jhi + pd.row_off;
    int32_t* off = a.off + pd.row_off;
    // each thread a run of consecutive rows: their checks and lengths, one scan
    // of the run totals, then the rows' offsets (the loads of a run are
    // independent, so they overlap instead of one block-wide round per 1024 rows)
    const int M = pd.M;
    const int per = (M + (int)blockDim.x - 1) / (int)blockDim.x;
    const int i0 = min(M, (int)threadIdx.x * per), i1 = min(M, i0 + per);
    // row i's cells on the path (0 for a row that breaks the staircase)
    auto row_len = [&](int i, int lo, int hi, int prev_hi) -> long long {
        bool ok = lo <= hi && lo >= 0 && hi < pd.N;
        if (i == 0) ok = ok && lo == 0;
        else ok = ok && (lo == prev_hi || lo == prev_hi + 1);
        if (i == M - 1) ok = ok && hi == pd.N - 1;
        return ok ? hi - lo + 1 : 0;
    };
    long long run = 0;
    const int hi0 = i0 > 0 && i0 < M ? jhi[i0 - 1] : 0;
    int prev_hi = hi0;
#pragma unroll 4
    for (int i = i0; i < i1; ++i) {
        const int lo = jlo[i], hi = jhi[i];
        const long long len = row_len(i, lo, hi, prev_hi);
        if (len == 0) set_error(a.ctl, ERR_PATH, i);
        run += len;
        prev_hi = hi;
    }
    long long tot;
    long long o = block_excl_scan(run, &tot);
    prev_hi = hi0;
#pragma unroll 4
    for (int i = i0; i < i1; ++i) {
        off[i] = (int32_t)o;
        const int lo = jlo[i], hi = jhi[i];
        o += row_len(i, lo, hi, prev_hi);
        prev_hi = hi;
    }
    if (threadIdx.x == 0) a.pres[pb].K = (int32_t)tot;
}

__global__ void assemble_scatter_kernel(AssembleArgs a) {
    const int pb = a.idx ? a.idx[blockIdx.y] : blockIdx.y;
    const PairDesc pd = a.pairs[pb];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pd.M) return;
    const int lo = a.jlo[pd.row_off + i], hi = a.jhi[pd.row_off + i];
    const long long o = a.off[pd.row_off + i];
    if (lo < 0 || hi < lo || o + (hi - lo) >= (long long)pd.M + pd.N - 1) return;
    for (int j = lo; j <= hi; ++j) {
        pd.path[2 * (o + j - lo)] = i;
        pd.path[2 * (o + j - lo) + 1] = j;
    }
}

cudaError_t launch_assemble(const AssembleArgs& a, cudaStream_t st) {
    assemble_scan_kernel<<<a.n_pairs, 1024, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 grid((a.max_M + 255) / 256, a.n_pairs);
    assemble_scatter_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

__global__ void fill_i32_kernel(int32_t* p, long long n, int32_t v) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        p[k] = v;
}

cudaError_t launch_fill_i32(int32_t* p, long long n, int32_t v, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long long g = (n + 255) / 256;
    fill_i32_kernel<<<(int)(g < 4096 ? g : 4096), 256, 0, st>>>(p, n, v);
    return cudaGetLastError();
}

// Node path of a local alignment: the global alignment of the substrings gives
// nodes relative to the start node; shift them to the whole problem's grid.
__global__ void offset_path_kernel(int32_t* p, long long K, int32_t da, int32_t db) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < K; t += (long long)gridDim.x * blockDim.x) {
        p[2 * t] += da;
        p[2 * t + 1] += db;
    }
}

cudaError_t launch_offset_path(int32_t* p, long long K, int32_t da, int32_t db, cudaStream_t st) {
    if (K <= 0) return cudaSuccess;
    long long g = (K + 255) / 256;
    offset_path_kernel<<<(int)(g < 4096 ? g : 4096), 256, 0, st>>>(p, K, da, db);
    return cudaGetLastError();
}

// Exactness guard of the int32 accumulator: every accumulated cost is at most
// max|x - y| * (M + N - 1), which must stay below 2^29.  Blocks of a 2-D grid
// (chunk, pair) reduce min and max of X and Y into minmax[4*pair..4*pair+3].
__global__ void int_range_kernel(const PairDesc* pairs, int32_t* minmax) {
    const PairDesc pd = pairs[blockIdx.y];
    int mn[2] = {INT_MAX, INT_MAX}, mx[2] = {INT_MIN, INT_MIN};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(pd.M, pd.N); i += gridDim.x * blockDim.x) {
        if (i < pd.M) {
            const int v = static_cast<const int32_t*>(pd.X)[i];
            mn[0] = min(mn[0], v);
            mx[0] = max(mx[0], v);
        }
        if (i < pd.N) {
            const int v = static_cast<const int32_t*>(pd.Y)[i];
            mn[1] = min(mn[1], v);
            mx[1] = max(mx[1], v);
        }
    }
    for (int o = 16; o; o >>= 1) {
        for (int t = 0; t < 2; ++t) {
            mn[t] = min(mn[t], __shfl_down_sync(kFull, mn[t], o));
            mx[t] = max(mx[t], __shfl_down_sync(kFull, mx[t], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        int32_t* r = minmax + 4 * blockIdx.y;
        atomicMin(r + 0, mn[0]);
        atomicMax(r + 1, mx[0]);
        atomicMin(r + 2, mn[1]);
        atomicMax(r + 3, mx[1]);
    }
}

__global__ void int_range_finish_kernel(const PairDesc* pairs, int n_pairs, const int32_t* minmax, LevelCtl* ctl,
                                        int32_t* pair_err) {
    for (int pb = blockIdx.x * blockDim.x + threadIdx.x; pb < n_pairs; pb += gridDim.x * blockDim.x) {
        const int32_t* r = minmax + 4 * pb;
        const long long c1 = (long long)r[1] - r[2], c2 = (long long)r[3] - r[0];
        const long long cmax = c1 > c2 ? c1 : c2;
        const bool bad = cmax * ((long long)pairs[pb].M + pairs[pb].N - 1) >= (1LL << 29);
        if (pair_err) pair_err[pb] = bad ? 1 : 0;
        else if (bad) set_error(ctl, ERR_OVERFLOW, pb);
    }
}

__global__ void minmax_init_kernel(int32_t* minmax, int n_pairs) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 4 * n_pairs; k += gridDim.x * blockDim.x)
        minmax[k] = (k & 1) ? INT_MIN : INT_MAX;
}

cudaError_t launch_int_range_check(const PairDesc* pairs, int n_pairs, int max_len, int32_t* minmax, LevelCtl* ctl,
                                   cudaStream_t st, int32_t* pair_err) {
    const int g0 = (4 * n_pairs + 255) / 256;
    minmax_init_kernel<<<g0 < 1024 ? g0 : 1024, 256, 0, st>>>(minmax, n_pairs);
    int gx = (max_len + 1023) / 1024;
    if (gx > 64) gx = 64;
    dim3 grid(gx < 1 ? 1 : gx, n_pairs);
    int_range_kernel<<<grid, 256, 0, st>>>(pairs, minmax);
    const int g1 = (n_pairs + 255) / 256;
    int_range_finish_kernel<<<g1 < 1024 ? g1 : 1024, 256, 0, st>>>(pairs, n_pairs, minmax, ctl, pair_err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- graph-driven level loop

__global__ void level_cond_kernel(LevelCtl* ctl, cudaGraphConditionalHandle h, int max_levels) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int lv = ++ctl->levels;
    const bool more = ctl->n_cur > 0 && ctl->err == ERR_NONE && lv < max_levels;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

cudaError_t launch_level_cond(LevelCtl* ctl, cudaGraphConditionalHandle h, int max_levels, cudaStream_t st) {
    level_cond_kernel<<<1, 32, 0, st>>>(ctl, h, max_levels);
    return cudaGetLastError();
}

// The level's sweep kernel (integer kinds): the one without tagged sweeps, whose
// band steps hold fewer registers, unless the plan found a tagged box.
__global__ void sweep_select_kernel(const LevelCtl* ctl, cudaGraphConditionalHandle h_plain,
                                    cudaGraphConditionalHandle h_tags) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const bool tags = ctl->n_tag > 0;
    cudaGraphSetConditional(h_plain, tags ? 0u : 1u);
    cudaGraphSetConditional(h_tags, tags ? 1u : 0u);
}

cudaError_t launch_sweep_select(const LevelCtl* ctl, cudaGraphConditionalHandle h_plain,
                                cudaGraphConditionalHandle h_tags, cudaStream_t st) {
    sweep_select_kernel<<<1, 32, 0, st>>>(ctl, h_plain, h_tags);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- serving support

__global__ void append_roots_kernel(const Box* roots, int n, Box* cur, int cur0, Box* base, int cap_base,
                                    long long base_area, LevelCtl* ctl) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int k = cur0;
    for (int r = 0; r < n; ++r) {
        const Box b = roots[r];
        if ((long long)b.H * b.W <= base_area) {
            const int j = ctl->n_base++;
            if (j < cap_base) base[j] = b;
            else set_error(ctl, ERR_CAPACITY, 3);
        } else {
            cur[k++] = b;
        }
    }
}

cudaError_t launch_append_roots(const Box* roots, int n, Box* cur, int cur0, Box* base, int cap_base,
                                long long base_area, LevelCtl* ctl, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    append_roots_kernel<<<1, 32, 0, st>>>(roots, n, cur, cur0, base, cap_base, base_area, ctl);
    return cudaGetLastError();
}

__global__ void mark_pairs_kernel(const Box* boxes, const LevelCtl* ctl, int32_t* flags) {
    const int n = ctl->n_cur;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) flags[boxes[i].pair] = 1;
}

cudaError_t launch_mark_pairs(const Box* boxes, const LevelCtl* ctl, int32_t* flags, cudaStream_t st) {
    mark_pairs_kernel<<<64, 256, 0, st>>>(boxes, ctl, flags);
    return cudaGetLastError();
}

}  // namespace dtwb
