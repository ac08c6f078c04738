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

// Partial minima of the window of split rows over one chunk of columns: for
// every row m, S = F + B - C (Lemma 2) minimised over the chunk, with the number
// of columns attaining the minimum and the lowest of them.  Block of 256 threads;
// rm[m] ends up with row m's merged values (rows m < nout).  A thread issues all
// loads of its column before it combines them (rows past the window repeat its
// last row and are dropped), so that one memory latency covers the column.
// LEAN (the sweep kernel's split phase, whose registers the band steps set): one
// split row at a time, nothing hoisted.
template <int KIND, int DIM, typename V, bool LEAN = false>
__device__ void chunk_minima(const SplitArgs& a, const Box& b, const PairDesc& pd, const Geom& g, const Sweep& fw,
                             const Sweep& bw, int q0, int q1, RowMin<V>* rm) {
    using Acc = typename AccOf<KIND>::T;
    __shared__ RowMin<V> s_part[kSplitRowsMax][8];
    // out rows are stored in each sweep's frame order (out_index): the backward
    // sweep's rows and columns run the other way
    const int nr = fw.nout, h = nr / 2;
    const Acc* F = static_cast<const Acc*>(a.outpool) + fw.out_off;
    const Acc* B = static_cast<const Acc*>(a.outpool) + bw.out_off;
    if constexpr (LEAN) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll 1
        for (int m = 0; m < nr; ++m) {
            RowMin<V> x{(V)0, 0, INT_MAX};
#pragma unroll 1
            for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
                int i, j;
                frame_to_global(b, g.axis, g.r - h + m, q, i, j);
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
            if (lane == 0) s_part[m][wid] = x;
        }
        __syncthreads();
        if (threadIdx.x < nr) {
            const int m = threadIdx.x;
            RowMin<V> x = s_part[m][0];
            for (int w = 1; w < nw; ++w) {
                const RowMin<V> y = s_part[m][w];
                x = (x.n == 0) ? y : (y.n == 0 ? x : merge(x, y));
            }
            rm[m] = x;
        }
        __syncthreads();
    } else {
    RowMin<V> part[kSplitRowsMax];
#pragma unroll
    for (int m = 0; m < kSplitRowsMax; ++m) part[m] = RowMin<V>{(V)0, 0, INT_MAX};
    // integer symbols are loaded with the rows; float frames row by row (their
    // registers)
    constexpr bool kHoist = int_kind(KIND);
    for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        V fb[kSplitRowsMax], cc[kSplitRowsMax];
#pragma unroll
        for (int m = 0; m < kSplitRowsMax; ++m) {
            const int mm = min(m, nr - 1);
            fb[m] = as_v<V>(F[out_index<Acc>(mm, q, nr)]) + as_v<V>(B[out_index<Acc>(nr - 1 - mm, g.Q - 1 - q, nr)]);
            if constexpr (kHoist) {
                int i, j;
                frame_to_global(b, g.axis, g.r - h + mm, q, i, j);
                cc[m] = (V)cell_cost<KIND, DIM>(pd, i, j, a.d);
            }
        }
#pragma unroll
        for (int m = 0; m < kSplitRowsMax; ++m) {
            if (m < nr) {
                V c;
                if constexpr (kHoist) {
                    c = cc[m];
                } else {
                    int i, j;
                    frame_to_global(b, g.axis, g.r - h + m, q, i, j);
                    c = (V)cell_cost<KIND, DIM>(pd, i, j, a.d);
                }
                const RowMin<V> x{fb[m] - c, 1, q};
                part[m] = part[m].n == 0 ? x : merge(part[m], x);
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int m = 0; m < nr; ++m) {
        RowMin<V> x = part[m];
        for (int o = 16; o; o >>= 1) {
            RowMin<V> y;
            y.v = __shfl_down_sync(kFull, x.v, o);
            y.n = __shfl_down_sync(kFull, x.n, o);
            y.q = __shfl_down_sync(kFull, x.q, o);
            if (lane + o < 32) x = (x.n == 0) ? y : (y.n == 0 ? x : merge(x, y));
        }
        if (lane == 0) s_part[m][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x < nr) {  // one thread per row
        const int m = threadIdx.x;
        RowMin<V> x = s_part[m][0];
        for (int w = 1; w < nw; ++w) {
            const RowMin<V> y = s_part[m][w];
            x = (x.n == 0) ? y : (y.n == 0 ? x : merge(x, y));
        }
        rm[m] = x;
    }
    __syncthreads();
    }
}

// The box's pivot from the minima of its split rows (thread 0 only), then its
// two children (or, when every split row tied on an integer box, the box itself
// again with split tags).
template <int KIND, int DIM, typename V>
__device__ void finish_box(const SplitArgs& a, const Box& b, const PairDesc& pd, const Geom& g, const Sweep& fw,
                           const Sweep& bw, int bi, const RowMin<V>* rm) {
    using Acc = typename AccOf<KIND>::T;
    int row = g.r, qs = 0;
    long long known_l = 0, known_r = 0, total_i = 0;
    double kl_f = 0, kr_f = 0, total_f = 0;
    bool retag = false;
    if (b.flags & BOX_TAG) {
        // canonical pivot: the tag that reached the box's last cell
        const SweepRes rr = a.res[2 * bi];
        qs = rr.end_tag;
        const Acc* out = static_cast<const Acc*>(a.outpool) + fw.out_off;  // one out row
        if (qs < 0 || qs >= g.Q) {
            set_error(a.ctl, ERR_CONSIST, 10);
            qs = 0;
        }
        int i, j;
        frame_to_global(b, g.axis, g.r, qs, i, j);
        const auto c = cell_cost<KIND, DIM>(pd, i, j, a.d);
        if constexpr (int_kind(KIND)) {
            total_i = rr.end_i;
            if (b.known_i >= 0 && b.known_i != total_i) set_error(a.ctl, ERR_CONSIST, 11);
            known_l = out[out_index<Acc>(0, qs, 1)];
            known_r = total_i - known_l + c;
        } else {
            total_f = rr.end_f;
            kl_f = as_v<double>(out[out_index<Acc>(0, qs, 1)]);
            kr_f = total_f - kl_f + (double)c;
        }
    } else {
        const int nr = fw.nout, h = nr / 2;
        const Acc* F = static_cast<const Acc*>(a.outpool) + fw.out_off;
        const Acc* B = static_cast<const Acc*>(a.outpool) + bw.out_off;
        // every split row's minimum is the box's optimal cost (Lemma 2)
        int pick = -1;
        if constexpr (int_kind(KIND)) {
            for (int m = 0; m < nr; ++m) {
                if (rm[m].v != rm[h].v) set_error(a.ctl, ERR_CONSIST, 12);
                if (b.known_i >= 0 && rm[m].v != b.known_i) set_error(a.ctl, ERR_CONSIST, 13);
            }
            // a row whose minimum is attained once: that cell is on every
            // optimal path, hence on the canonical one; nearest the middle first
            for (int k = 0; k <= h && pick < 0; ++k) {
                if (rm[h - k].n == 1) pick = h - k;
                else if (rm[h + k].n == 1) pick = h + k;
            }
            total_i = rm[h].v;
        } else {
            pick = h;  // any minimiser gives an optimal path (float kind)
            total_f = rm[h].v;
        }
        if (pick < 0) {
            retag = true;
        } else {
            row = g.r - h + pick;
            qs = rm[pick].q;
            if constexpr (int_kind(KIND)) {
                known_l = F[out_index<Acc>(pick, qs, nr)];
                known_r = B[out_index<Acc>(nr - 1 - pick, g.Q - 1 - qs, nr)];
            } else {
                kl_f = as_v<double>(F[out_index<Acc>(pick, qs, nr)]);
                kr_f = as_v<double>(B[out_index<Acc>(nr - 1 - pick, g.Q - 1 - qs, nr)]);
            }
        }
    }
    if (b.flags & BOX_ROOT) {
        a.pres[b.pair].cost_i = total_i;
        a.pres[b.pair].cost_f = total_f;
    }
    if constexpr (KIND == KIND_EDIT) {
        // a child's sweeps carry the symbols' costs at its own corners, which
        // differ from the parent's: its optimum is not checked against them
        known_l = -1;
        known_r = -1;
    }
    if (retag) {  // every split row tied: sweep this box again with split tags
        Box t = b;
        t.flags = BOX_TAG;
        t.known_i = KIND == KIND_EDIT ? -1 : total_i;  // edit: the tag sweep's end carries no backward corner term
        atomicAdd((unsigned long long*)&a.ctl->retag, 1ULL);
        emit_child(a, t);
    } else {
        Box L = b, Rb = b;
        L.flags = 0;
        Rb.flags = 0;
        if (g.axis == 0) {
            L.H = row + 1;
            L.W = qs + 1;
            Rb.i0 = b.i0 + row;
            Rb.j0 = b.j0 + qs;
            Rb.H = b.H - row;
            Rb.W = b.W - qs;
        } else {
            L.H = qs + 1;
            L.W = row + 1;
            Rb.i0 = b.i0 + qs;
            Rb.j0 = b.j0 + row;
            Rb.H = b.H - qs;
            Rb.W = b.W - row;
        }
        L.known_i = known_l;
        Rb.known_i = known_r;
        L.known_f = kl_f;
        Rb.known_f = kr_f;
        emit_child(a, L);
        emit_child(a, Rb);
    }
}


// Progress words of a sweep's split rows, read by fused split items (four ints
// per sweep, reset by the plan): [0] and [1] column blocks whose split (out) rows
// the first and second band holding them have stored ([1] starts complete when
// one band holds them all), [2] set once the band holding the sweep's last row
// has recorded its last cell.
constexpr int kProgWords = 4;

// Waits (thread 0, bounded, backing off) until *p >= target; gpu-scope acquire.
__device__ __forceinline__ void wait_prog(const int* p, int target, LevelCtl* ctl, int spin_limit) {
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

// One split work item (block-wide): item it of the level -- a column chunk of a
// box's split rows, or a tagged box whole.  Its partial minima are written; the
// item that finishes a box last merges them and emits the box's children.
// prog != nullptr (the sweep kernel's split phase, sweeps still running): the
// item first waits until both half sweeps have stored its columns' split rows
// (U columns per block).
template <int KIND, int DIM, bool LEAN = false>
__device__ void split_item(const SplitArgs& a, int it, int U, const int* prog, int spin_limit = 1 << 22) {
    using V = typename std::conditional<int_kind(KIND), long long, double>::type;
    __shared__ RowMin<V> rm[kSplitRowsMax];
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
    const int chunk = it - fw.item0, nitems = fw.nitems;
    const int q0 = chunk * kSplitChunk, q1 = min(q0 + kSplitChunk, g.Q);
    if (prog != nullptr && threadIdx.x == 0) {
        const int* pf = prog + (size_t)(2 * bi) * kProgWords;
        if (b.flags & BOX_TAG) {
            wait_prog(pf, fw.nblk, a.ctl, spin_limit);
            wait_prog(pf + 1, fw.nblk, a.ctl, spin_limit);
            wait_prog(pf + 2, 1, a.ctl, spin_limit);
        } else {
            // forward rows over columns [q0, q1); backward rows over the mirrored columns
            const int* pb = prog + (size_t)(2 * bi + 1) * kProgWords;
            const int nf = (q1 - 1) / U + 1, nb = (g.Q - 1 - q0) / U + 1;
            wait_prog(pf, nf, a.ctl, spin_limit);
            wait_prog(pf + 1, nf, a.ctl, spin_limit);
            wait_prog(pb, nb, a.ctl, spin_limit);
            wait_prog(pb + 1, nb, a.ctl, spin_limit);
        }
    }
    if (prog != nullptr) __syncthreads();
    if (b.flags & BOX_TAG) {
        if (threadIdx.x == 0) finish_box<KIND, DIM, V>(a, b, pd, g, fw, bw, bi, rm);
        __syncthreads();
        return;
    }
    chunk_minima<KIND, DIM, V, LEAN>(a, b, pd, g, fw, bw, q0, q1, rm);
    const int nr = fw.nout;
    if (nitems > 1 && threadIdx.x < nr) {  // each writer fences its own row
        partials[(size_t)it * kSplitRowsMax + threadIdx.x] = rm[threadIdx.x];
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) s_last = nitems == 1 || atomicAdd(&a.box_done[bi], 1) == nitems - 1;
    __syncthreads();
    if (s_last && nitems > 1) {
        // merge the box's partial minima: one warp per split row, lanes over items
        __threadfence();
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int m = wid; m < nr; m += nw) {
            RowMin<V> x{(V)0, 0, INT_MAX};
            for (int k = lane; k < nitems; k += 32) {
                const RowMin<V> y = partials[(size_t)(fw.item0 + k) * kSplitRowsMax + m];
                x = (x.n == 0) ? y : (y.n == 0 ? x : merge(x, y));
            }
            for (int o = 16; o; o >>= 1) {
                RowMin<V> y;
                y.v = __shfl_down_sync(kFull, x.v, o);
                y.n = __shfl_down_sync(kFull, x.n, o);
                y.q = __shfl_down_sync(kFull, x.q, o);
                if (lane + o < 32) x = (x.n == 0) ? y : (y.n == 0 ? x : merge(x, y));
            }
            if (lane == 0) rm[m] = x;
        }
        __syncthreads();
    }
    if (s_last && threadIdx.x == 0) finish_box<KIND, DIM, V>(a, b, pd, g, fw, bw, bi, rm);
    __syncthreads();
}

}  // namespace dtwb
