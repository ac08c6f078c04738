// The split of Algorithm 2 (Lemmas 1 and 2): the device code shared by the
// level's split kernel and by the sweep kernel's split phase (blocks that have
// finished their sweep tickets take split work items while the window bands
// are still running).  Internal header.
#pragma once

#include <climits>
#include <type_traits>

#include "dtw_common.cuh"
#include "dtw_kernels.h"

namespace dtwb {

// ---------------------------------------------------------------- geometry

// Split geometry of a box: the longer side is cut at its middle index (a row
// split when H >= W).  Frame rows p run along the cut side.
struct Geom {
    int axis, P, Q, r;
};

__device__ __forceinline__ Geom geom_of(const Box& b) {
    Geom g;
    g.axis = b.H >= b.W ? 0 : 1;
    g.P = g.axis ? b.W : b.H;
    g.Q = g.axis ? b.H : b.W;
    g.r = (g.P - 1) / 2;
    return g;
}

// global (i, j) of frame cell (p, q) of a forward sweep
__device__ __forceinline__ void frame_to_global(const Box& b, int axis, int p, int q, int& i, int& j) {
    if (axis == 0) {
        i = b.i0 + p;
        j = b.j0 + q;
    } else {
        i = b.i0 + q;
        j = b.j0 + p;
    }
}

// ---------------------------------------------------------------- split

__device__ __forceinline__ void emit_child(const SplitArgs& a, const Box& c) {
    const long long area = (long long)c.H * c.W;
    if (area <= a.base_area && !(c.flags & BOX_TAG)) {
        const int k = atomicAdd(&a.ctl->n_base, 1);
        if (k < a.cap_base) a.base[k] = c;
        else set_error(a.ctl, ERR_CAPACITY, 1);
    } else {
        const int k = atomicAdd(&a.ctl->n_next, 1);
        if (k < a.cap_next) a.next[k] = c;
        else set_error(a.ctl, ERR_CAPACITY, 2);
    }
}

// (min, number of columns attaining it, lowest such column) of one split row
template <typename V>
struct RowMin {
    V v;
    int n, q;
};

template <typename V>
__device__ __forceinline__ RowMin<V> merge(RowMin<V> x, RowMin<V> y) {
    if (y.v < x.v) return y;
    if (x.v < y.v) return x;
    return RowMin<V>{x.v, x.n + y.n, min(x.q, y.q)};
}

// An accumulator as the split's comparison type (exact for every kind).
template <typename V, typename A>
__device__ __forceinline__ V as_v(A x) {
    if constexpr (std::is_same<A, DF>::value) return (V)to_double(x);
    else return (V)x;
}

// Partial minima of window t of split rows over one chunk of columns: for every
// row e of the window, S = F + B - C (Lemma 2) minimised over the chunk, with the
// number of columns attaining the minimum and the lowest of them.  Block of 256
// threads (or the sweep kernel's block); rm[e] ends up with row e's merged values
// (e < owin).  A thread issues all loads of its column before it combines them
// (rows past the window repeat its last row and are dropped), so that one memory
// latency covers the column.  LEAN (the sweep kernel's split phase, whose
// registers the band steps set): one split row at a time, nothing hoisted.
template <int KIND, int DIM, typename V, bool LEAN = false>
__device__ void chunk_minima(const SplitArgs& a, const Box& b, const PairDesc& pd, const Geom& g, const Sweep& fw,
                             const Sweep& bw, int t, int q0, int q1, RowMin<V>* rm) {
    using Acc = typename AccOf<KIND>::T;
    __shared__ RowMin<V> s_part[kSplitRowsMax][8];
    // out rows are stored in each sweep's frame order (out_index): the backward
    // sweep's rows and columns run the other way; out row m of the forward sweep
    // is out row nr-1-m of the backward one
    const int nr = fw.nout, ow = fw.owin, m0 = t * ow;
    const int p0 = out_frame_row(fw, m0);  // frame row of the window's first row
    const Acc* F = static_cast<const Acc*>(a.outpool) + fw.out_off;
    const Acc* B = static_cast<const Acc*>(a.outpool) + bw.out_off;
    if constexpr (LEAN) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll 1
        for (int e = 0; e < ow; ++e) {
            const int m = m0 + e;
            RowMin<V> x{(V)0, 0, INT_MAX};
#pragma unroll 1
            for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
                int i, j;
                frame_to_global(b, g.axis, p0 + e, q, i, j);
                const V s = as_v<V>(F[out_index<Acc>(m, q, nr)]) + as_v<V>(B[out_index<Acc>(nr - 1 - m, g.Q - 1 - q, nr)]) -
                            (V)cell_cost<KIND, DIM>(pd, i, j, a.d);
                const RowMin<V> y{s, 1, q};
                x = x.n == 0 ? y : merge(x, y);
            }
            for (int o = 16; o; o >>= 1) {
                RowMin<V> y;
                y.v = __shfl_down_sync(kFull, x.v, o);
                y.n = __shfl_down_sync(kFull, x.n, o);
                y.q = __shfl_down_sync(kFull, x.q, o);
                if (lane + o < 32) x = (x.n == 0) ? y : (y.n == 0 ? x : merge(x, y));
            }
            if (lane == 0) s_part[e][wid] = x;
        }
        __syncthreads();
        if (threadIdx.x < ow) {
            const int e = threadIdx.x;
            RowMin<V> x = s_part[e][0];
            for (int w = 1; w < nw; ++w) {
                const RowMin<V> y = s_part[e][w];
                x = (x.n == 0) ? y : (y.n == 0 ? x : merge(x, y));
            }
            rm[e] = x;
        }
        __syncthreads();
    } else {
    RowMin<V> part[kSplitRowsMax];
#pragma unroll
    for (int e = 0; e < kSplitRowsMax; ++e) part[e] = RowMin<V>{(V)0, 0, INT_MAX};
    // integer symbols are loaded with the rows; float frames row by row (their
    // registers)
    constexpr bool kHoist = int_kind(KIND);
    for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        V fb[kSplitRowsMax], cc[kSplitRowsMax];
#pragma unroll
        for (int e = 0; e < kSplitRowsMax; ++e) {
            const int ee = min(e, ow - 1), m = m0 + ee;
            fb[e] = as_v<V>(F[out_index<Acc>(m, q, nr)]) + as_v<V>(B[out_index<Acc>(nr - 1 - m, g.Q - 1 - q, nr)]);
            if constexpr (kHoist) {
                int i, j;
                frame_to_global(b, g.axis, p0 + ee, q, i, j);
                cc[e] = (V)cell_cost<KIND, DIM>(pd, i, j, a.d);
            }
        }
#pragma unroll
        for (int e = 0; e < kSplitRowsMax; ++e) {
            if (e < ow) {
                V c;
                if constexpr (kHoist) {
                    c = cc[e];
                } else {
                    int i, j;
                    frame_to_global(b, g.axis, p0 + e, q, i, j);
                    c = (V)cell_cost<KIND, DIM>(pd, i, j, a.d);
                }
                const RowMin<V> x{fb[e] - c, 1, q};
                part[e] = part[e].n == 0 ? x : merge(part[e], x);
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int e = 0; e < ow; ++e) {
        RowMin<V> x = part[e];
        for (int o = 16; o; o >>= 1) {
            RowMin<V> y;
            y.v = __shfl_down_sync(kFull, x.v, o);
            y.n = __shfl_down_sync(kFull, x.n, o);
            y.q = __shfl_down_sync(kFull, x.q, o);
            if (lane + o < 32) x = (x.n == 0) ? y : (y.n == 0 ? x : merge(x, y));
        }
        if (lane == 0) s_part[e][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < ow) {  // one thread per row
        const int e = threadIdx.x;
        RowMin<V> x = s_part[e][0];
        for (int w = 1; w < nw; ++w) {
            const RowMin<V> y = s_part[e][w];
            x = (x.n == 0) ? y : (y.n == 0 ? x : merge(x, y));
        }
        rm[e] = x;
    }
    __syncthreads();
    }
}

// The box's pivots from the minima of its split rows, then its children: the
// pieces between consecutive pivots (or, when no split row of an integer box has
// a unique minimiser, the box itself again with split tags).  Called by every
// thread of the block: one thread per window picks its pivot and loads its
// forward and backward values, thread 0 orders the pivots and forms the pieces,
// one thread per piece emits it.
//
// Every split row's minimum of F + B - C is the box's optimum and every cell
// attaining it lies on an optimal path (Lemma 2); a cell that attains it alone
// lies on every optimal path.  Integer kind: per window the row nearest its
// centre whose minimum is attained once -- all such cells lie on the canonical
// path, so they are consistent and the pieces between them keep it.  Float
// kind: the middle window's centre row (any minimiser: some optimal path) and
// the other windows' centre rows whose minimum is attained once (on every
// optimal path, so on that one too); a pivot that would break the monotone
// order (possible only through rounding) is dropped.
template <int KIND, int DIM, typename V>
__device__ void finish_box(const SplitArgs& a, const Box& b, const PairDesc& pd, const Geom& g, const Sweep& fw,
                           const Sweep& bw, int bi, const RowMin<V>* rm) {
    using Acc = typename AccOf<KIND>::T;
    __shared__ int s_m[kSplitWinMax];  // per window: its pivot's out row, or -1
    __shared__ int s_q[kSplitWinMax];
    __shared__ V s_f[kSplitWinMax];    // forward value at the pivot
    __shared__ V s_b[kSplitWinMax];    // backward value at the pivot
    __shared__ V s_c[kSplitWinMax];    // the pivot cell's cost
    __shared__ Box s_child[kSplitWinMax + 1];
    __shared__ int s_nchild;
    const int tid = threadIdx.x;
    const Acc* F = static_cast<const Acc*>(a.outpool) + fw.out_off;
    const Acc* B = static_cast<const Acc*>(a.outpool) + bw.out_off;
    const bool tag = (b.flags & BOX_TAG) != 0;
    const int nr = fw.nout, ow = fw.owin, nw = tag ? 1 : fw.onw, h = ow / 2, cw = (nw - 1) / 2;
    const int mid = cw * ow + h;  // the middle split row
    if (!tag) {
        // every split row's minimum is the box's optimal cost (Lemma 2)
        if constexpr (int_kind(KIND)) {
            for (int m = tid; m < nr; m += blockDim.x) {
                if (rm[m].v != rm[mid].v) set_error(a.ctl, ERR_CONSIST, 12);
                if (b.known_i >= 0 && rm[m].v != b.known_i) set_error(a.ctl, ERR_CONSIST, 13);
            }
        }
        if (tid < nw) {
            const int t = tid;
            int pick = -1;
            if constexpr (int_kind(KIND)) {
                for (int k = 0; k <= h && pick < 0; ++k) {
                    if (rm[t * ow + h - k].n == 1) pick = t * ow + h - k;
                    else if (rm[t * ow + h + k].n == 1) pick = t * ow + h + k;
                }
            } else {
                if (t == cw || rm[t * ow + h].n == 1) pick = t * ow + h;
            }
            s_m[t] = pick;
            if (pick >= 0) {
                const int q = rm[pick].q, p = out_frame_row(fw, pick);
                int i, j;
                frame_to_global(b, g.axis, p, q, i, j);
                s_q[t] = q;
                s_f[t] = as_v<V>(F[out_index<Acc>(pick, q, nr)]);
                s_b[t] = as_v<V>(B[out_index<Acc>(nr - 1 - pick, g.Q - 1 - q, nr)]);
                s_c[t] = (V)cell_cost<KIND, DIM>(pd, i, j, a.d);
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        // corners of the pieces in frame coordinates (p, q): the box's first
        // cell, the pivots, its last cell; per piece the known optimum
        int cp[kSplitWinMax + 2], cq[kSplitWinMax + 2];
        V kv[kSplitWinMax + 1];
        int npiv = 0;
        V total = 0;
        bool retag = false;
        cp[0] = 0;
        cq[0] = 0;
        if (tag) {
            // canonical pivot: the tag that reached the box's last cell
            const SweepRes rr = a.res[2 * bi];
            int qs = rr.end_tag;
            if (qs < 0 || qs >= g.Q) {
                set_error(a.ctl, ERR_CONSIST, 10);
                qs = 0;
            }
            int i, j;
            frame_to_global(b, g.axis, g.r, qs, i, j);
            const V c = (V)cell_cost<KIND, DIM>(pd, i, j, a.d);
            npiv = 1;
            cp[1] = g.r;
            cq[1] = qs;
            if constexpr (int_kind(KIND)) {
                total = rr.end_i;
                if (b.known_i >= 0 && b.known_i != total) set_error(a.ctl, ERR_CONSIST, 11);
            } else {
                total = rr.end_f;
            }
            kv[0] = as_v<V>(F[out_index<Acc>(0, qs, 1)]);  // one out row
            kv[1] = total - kv[0] + c;
        } else {
            total = rm[mid].v;
            // columns never decrease along a warping path: keep the pivots that
            // agree with the anchor (float kind: the middle window's; integer
            // kind: the first pivot -- they all agree)
            int anchor = -1;
            for (int t = 0; t < nw && anchor < 0; ++t)
                if (s_m[t] >= 0 && (int_kind(KIND) || t == cw)) anchor = t;
            if (anchor < 0) {
                retag = true;
            } else {
                bool keep[kSplitWinMax];
                for (int t = 0; t < nw; ++t) keep[t] = false;
                keep[anchor] = true;
                for (int t = anchor - 1, qq = s_q[anchor]; t >= 0; --t) {
                    if (s_m[t] < 0) continue;
                    if (s_q[t] <= qq) {
                        keep[t] = true;
                        qq = s_q[t];
                    } else if (int_kind(KIND)) {
                        set_error(a.ctl, ERR_CONSIST, 14);
                    }
                }
                for (int t = anchor + 1, qq = s_q[anchor]; t < nw; ++t) {
                    if (s_m[t] < 0) continue;
                    if (s_q[t] >= qq) {
                        keep[t] = true;
                        qq = s_q[t];
                    } else if (int_kind(KIND)) {
                        set_error(a.ctl, ERR_CONSIST, 14);
                    }
                }
                // piece k runs from the previous corner to pivot k: its optimum is
                // the forward value there minus the one before the previous pivot;
                // the last piece's is the backward value at the last pivot
                V fprev = 0;
                int last = -1;
                for (int t = 0; t < nw; ++t) {
                    if (!keep[t]) continue;
                    cp[npiv + 1] = out_frame_row(fw, s_m[t]);
                    cq[npiv + 1] = s_q[t];
                    kv[npiv] = s_f[t] - fprev;
                    fprev = s_f[t] - s_c[t];
                    last = t;
                    ++npiv;
                }
                kv[npiv] = s_b[last];
            }
        }
        if (b.flags & BOX_ROOT) {
            if constexpr (int_kind(KIND)) a.pres[b.pair].cost_i = (long long)total;
            else a.pres[b.pair].cost_f = (double)total;
        }
        if (retag) {  // no split row with a unique minimiser: sweep this box again with split tags
            Box t = b;
            t.flags = BOX_TAG;
            t.known_i = KIND == KIND_EDIT ? -1 : (long long)total;  // edit: the tag sweep's end carries no backward corner term
            atomicAdd((unsigned long long*)&a.ctl->retag, 1ULL);
            s_child[0] = t;
            s_nchild = 1;
        } else {
            cp[npiv + 1] = g.P - 1;
            cq[npiv + 1] = g.Q - 1;
            for (int k = 0; k <= npiv; ++k) {
                Box c = b;
                c.flags = 0;
                const int ph = cp[k + 1] - cp[k] + 1, qw = cq[k + 1] - cq[k] + 1;
                if (g.axis == 0) {
                    c.i0 = b.i0 + cp[k];
                    c.j0 = b.j0 + cq[k];
                    c.H = ph;
                    c.W = qw;
                } else {
                    c.i0 = b.i0 + cq[k];
                    c.j0 = b.j0 + cp[k];
                    c.H = qw;
                    c.W = ph;
                }
                // edit distance: a child's sweeps carry the symbols' costs at its own
                // corners, which differ from the parent's: its optimum is not checked
                if constexpr (int_kind(KIND)) c.known_i = KIND == KIND_EDIT ? -1 : (long long)kv[k];
                else c.known_i = -1;
                c.known_f = int_kind(KIND) ? (double)NAN : (double)kv[k];
                s_child[k] = c;
            }
            s_nchild = npiv + 1;
        }
    }
    __syncthreads();
    if (tid < s_nchild) emit_child(a, s_child[tid]);
    __syncthreads();
}


// Progress words of a sweep's split rows, read by fused split items (four ints
// per sweep, reset by the plan): [0] bands holding split rows that have stored
// them all, [1] how many bands hold split rows, [2] set once the band holding the
// sweep's last row has recorded its last cell.
constexpr int kProgWords = 4;

// Waits (thread 0, bounded, backing off) until p[0] >= p[1], or with target >= 0
// until p[0] >= target; gpu-scope acquire.
__device__ __forceinline__ void wait_prog(const int* p, int target, LevelCtl* ctl, int spin_limit) {
    if (target < 0) target = ld_relaxed(p + 1);
    unsigned nap = 32;
    for (int it = 0;; ++it) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
        if (v >= target) return;
        if (it >= spin_limit || ((it & 63) == 63 && ld_relaxed(&ctl->err) != ERR_NONE)) {
            set_error(ctl, ERR_TIMEOUT, -3);
            return;
        }
        __nanosleep(nap);
        nap = nap < 1024 ? 2 * nap : 1024;
    }
}

// One split work item (block-wide): item it of the level -- a column chunk of one
// window of a box's split rows, or a tagged box whole.  Its partial minima are
// written; the item that finishes a box last merges them and emits the box's
// children.  prog != nullptr (the sweep kernel's split phase, sweeps still
// running): the item first waits until the bands holding the split rows of both
// half sweeps have ended.
template <int KIND, int DIM, bool LEAN = false>
__device__ void split_item(const SplitArgs& a, int it, const int* prog, int spin_limit = 1 << 22) {
    // the comparison type: F + B - C is below 2^30 for the integer kinds (the
    // accumulators' exactness guard keeps F and B below 2^29)
    using V = typename std::conditional<int_kind(KIND), int32_t, double>::type;
    __shared__ RowMin<V> rm[kOutRowsMax];
    __shared__ int s_last, s_box;
    RowMin<V>* partials = static_cast<RowMin<V>*>(a.partials);
    const int n_boxes = a.n_boxes >= 0 ? a.n_boxes : a.ctl->n_cur;
    // the box of item it: the last box whose first item is <= it (item0 rises
    // with the box index).  Up to 8 boxes a thread, the block tests every box at
    // once; beyond that, a binary search.
    int bi;
    if (n_boxes <= 8 * (int)blockDim.x) {
        if (threadIdx.x == 0) s_box = 0;
        __syncthreads();
        int first[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int x = threadIdx.x + k * blockDim.x;
            first[k] = x < n_boxes ? a.sweeps[2 * x].item0 : INT_MAX;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int x = threadIdx.x + k * blockDim.x;
            if (first[k] <= it) atomicMax(&s_box, x);
        }
        __syncthreads();
        bi = s_box;
    } else {
        int lo = 0, hi = n_boxes - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.sweeps[2 * mid].item0 <= it) lo = mid;
            else hi = mid - 1;
        }
        bi = lo;
    }
    const Box b = a.boxes[bi];
    const PairDesc pd = a.pairs[b.pair];
    const Geom g = geom_of(b);
    const Sweep& fw = a.sweeps[2 * bi];
    const Sweep& bw = a.sweeps[2 * bi + 1];
    // item k of the box: window k / nch, column chunk k % nch
    const int ic = split_item_cols(fw.onw);
    const int nch = (g.Q + ic - 1) / ic;
    const int k = it - fw.item0, nitems = fw.nitems;
    const int t = k / nch, chunk = k - t * nch;
    const int q0 = chunk * ic, q1 = min(q0 + ic, g.Q);
    if (prog != nullptr && threadIdx.x == 0) {
        const int* pf = prog + (size_t)(2 * bi) * kProgWords;
        wait_prog(pf, -1, a.ctl, spin_limit);
        if (b.flags & BOX_TAG) wait_prog(pf + 2, 1, a.ctl, spin_limit);
        else wait_prog(prog + (size_t)(2 * bi + 1) * kProgWords, -1, a.ctl, spin_limit);
    }
    if (prog != nullptr) __syncthreads();
    if (b.flags & BOX_TAG) {
        finish_box<KIND, DIM, V>(a, b, pd, g, fw, bw, bi, rm);
        return;
    }
    const int ow = fw.owin, nr = fw.nout;
    chunk_minima<KIND, DIM, V, LEAN>(a, b, pd, g, fw, bw, t, q0, q1, rm + t * ow);
    if (nitems > 1 && threadIdx.x < ow) {  // each writer fences its own row
        partials[(size_t)it * kSplitRowsMax + threadIdx.x] = rm[t * ow + threadIdx.x];
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) s_last = nitems == 1 || atomicAdd(&a.box_done[bi], 1) == nitems - 1;
    __syncthreads();
    if (s_last && nitems > 1) {
        // merge the box's partial minima: a group of gs threads per split row
        // (gs a power of two, every row in one pass where the block allows),
        // its threads over the row's window's column chunks
        __threadfence();
        int gs = 32;
        while (gs > 1 && gs * nr > (int)blockDim.x) gs >>= 1;
        const int per = (int)blockDim.x / gs, sub = (int)threadIdx.x % gs;
        for (int m0 = 0; m0 < nr; m0 += per) {  // the same count of passes for every thread
            const int m = m0 + (int)threadIdx.x / gs;
            RowMin<V> x{(V)0, 0, INT_MAX};
            if (m < nr) {
                const int tt = m / ow, e = m - tt * ow;
                for (int c = sub; c < nch; c += gs) {
                    const RowMin<V> y = partials[(size_t)(fw.item0 + tt * nch + c) * kSplitRowsMax + e];
                    x = (x.n == 0) ? y : (y.n == 0 ? x : merge(x, y));
                }
            }
            for (int o = gs >> 1; o; o >>= 1) {
                RowMin<V> y;
                y.v = __shfl_down_sync(kFull, x.v, o);
                y.n = __shfl_down_sync(kFull, x.n, o);
                y.q = __shfl_down_sync(kFull, x.q, o);
                if (sub + o < gs) x = (x.n == 0) ? y : (y.n == 0 ? x : merge(x, y));
            }
            if (m < nr && sub == 0) rm[m] = x;
        }
        __syncthreads();
    }
    if (s_last) finish_box<KIND, DIM, V>(a, b, pd, g, fw, bw, bi, rm);
}

}  // namespace dtwb
