// Per-level kernels of the divide-and-conquer recursion (Section 3.2,
// Algorithm 2): planning the sweeps of every box of a level, choosing each box's
// pivot on its split row (Lemmas 1 and 2), emitting the two child boxes that
// share the pivot, finishing small boxes with a full-table DP and backtrace
// (Section 2.1), and assembling the per-pair warping paths.
#include <climits>

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

// ---------------------------------------------------------------- plan

// One block of 1024 threads.  For every box of the level: its sweeps (one
// tagged forward sweep, or a forward half and a backward half, or one full
// forward sweep), their band tickets and pool offsets; then the level counters.
__global__ void __launch_bounds__(1024) plan_kernel(PlanArgs a) {
    __shared__ long long carry[3];
    __shared__ unsigned long long cells_sh[2];
    const int nsw = a.mode == MODE_FB ? 2 : 1;
    if (threadIdx.x < 3) carry[threadIdx.x] = 0;
    if (threadIdx.x < 2) cells_sh[threadIdx.x] = 0;
    __syncthreads();
    unsigned long long my_cells = 0, my_tag = 0;
    for (int base = 0; base < a.n_boxes * nsw; base += blockDim.x) {
        const int s = base + threadIdx.x;
        const bool valid = s < a.n_boxes * nsw;
        Sweep sw = {};
        long long nb = 0, nbuf = 0, nout = 0;
        if (valid) {
            const int bi = s / nsw, dir = s % nsw;
            const Box b = a.boxes[bi];
            const PairDesc pd = a.pairs[b.pair];
            const Geom g = geom_of(b);
            sw.box = bi;
            sw.dir = dir;
            sw.axis = g.axis;
            sw.Q = g.Q;
            sw.nblk = (g.Q + a.U - 1) / a.U;
            if (a.mode == MODE_TAG) {
                sw.rows = g.P;
                sw.out_row = g.r;
                sw.tag_row = g.r;
            } else if (a.mode == MODE_FB) {
                sw.rows = dir == 0 ? g.r + 1 : g.P - g.r;
                sw.out_row = sw.rows - 1;  // both halves end on the split row
                sw.tag_row = -1;
            } else {
                sw.rows = g.P;
                sw.out_row = -1;
                sw.tag_row = -1;
            }
            sw.nbands = (sw.rows + a.BR - 1) / a.BR;
            sw.rowseq = g.axis ? pd.Y : pd.X;
            sw.colseq = g.axis ? pd.X : pd.Y;
            const int rb0 = g.axis ? b.j0 : b.i0, rlen = g.axis ? b.W : b.H;
            const int cb0 = g.axis ? b.i0 : b.j0, clen = g.axis ? b.H : b.W;
            if (dir == 0) {
                sw.rbase = rb0;
                sw.rstep = 1;
                sw.cbase = cb0;
                sw.cstep = 1;
            } else {  // the reversed series X_R, Y_R of Algorithm 2
                sw.rbase = rb0 + rlen - 1;
                sw.rstep = -1;
                sw.cbase = cb0 + clen - 1;
                sw.cstep = -1;
            }
            nb = sw.nbands;
            nbuf = (long long)sw.nblk * a.U;
            nout = a.mode == MODE_COST ? 0 : g.Q;
            my_cells += (unsigned long long)sw.rows * (unsigned long long)g.Q;
            if (sw.tag_row >= 0) my_tag += (unsigned long long)(sw.rows - sw.tag_row) * g.Q;
        }
        long long t0, t1, t2;
        const long long e0 = block_excl_scan(nb, &t0);
        const long long e1 = block_excl_scan(nbuf, &t1);
        const long long e2 = block_excl_scan(nout, &t2);
        if (valid) {
            sw.band_begin = carry[0] + e0;
            sw.prog_off = carry[0] + e0;
            sw.buf_off = carry[1] + e1;
            sw.out_off = carry[2] + e2;
            if (s < a.cap_sweeps) a.sweeps[s] = sw;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry[0] += t0;
            carry[1] += t1;
            carry[2] += t2;
        }
        __syncthreads();
    }
    atomicAdd(&cells_sh[0], my_cells);
    atomicAdd(&cells_sh[1], my_tag);
    __syncthreads();
    const long long total_bands = carry[0];
    const bool fits = (long long)a.n_boxes * nsw <= a.cap_sweeps && carry[1] <= a.cap_buf &&
                      carry[2] <= a.cap_out && total_bands <= a.cap_prog;
    for (long long k = threadIdx.x; k < (fits ? total_bands : 0); k += blockDim.x) a.progpool[k] = 0;
    if (threadIdx.x == 0) {
        LevelCtl* c = a.ctl;
        c->ticket = 0;
        c->n_next = 0;
        c->need_buf = carry[1];
        c->need_prog = total_bands;
        if (fits) {
            c->n_sweeps = a.n_boxes * nsw;
            c->n_tickets = total_bands;
            c->sweep_cells += cells_sh[0];
            c->tag_cells += cells_sh[1];
        } else {
            c->n_sweeps = 0;
            c->n_tickets = 0;
            set_error(c, ERR_CAPACITY, 0);
        }
    }
}

cudaError_t launch_plan(const PlanArgs& a, cudaStream_t st) {
    plan_kernel<<<1, 1024, 0, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- split

__device__ __forceinline__ void emit_child(const SplitArgs& a, const Box& c) {
    const long long area = (long long)c.H * c.W;
    if (area <= a.base_area) {
        const int k = atomicAdd(&a.ctl->n_base, 1);
        if (k < a.cap_base) a.base[k] = c;
        else set_error(a.ctl, ERR_CAPACITY, 1);
    } else {
        const int k = atomicAdd(&a.ctl->n_next, 1);
        if (k < a.cap_next) a.next[k] = c;
        else set_error(a.ctl, ERR_CAPACITY, 2);
    }
}

template <int KIND, int DIM>
__device__ void split_box(const SplitArgs& a, int bi) {
    using Acc = typename AccOf<KIND>::T;
    __shared__ double s_val[32];
    __shared__ long long s_ival[32];
    __shared__ int s_q[32];
    const Box b = a.boxes[bi];
    const PairDesc pd = a.pairs[b.pair];
    const Geom g = geom_of(b);
    int qs = 0;
    long long known_l = 0, known_r = 0, total_i = 0;
    double kl_f = 0, kr_f = 0, total_f = 0;
    if (a.mode == MODE_TAG) {
        // canonical pivot: the tag that reached the box's last cell
        if (threadIdx.x == 0) {
            const Sweep& sw = a.sweeps[bi];
            const SweepRes rr = a.res[bi];
            qs = rr.end_tag;
            const Acc* out = static_cast<const Acc*>(a.outpool) + sw.out_off;
            if (qs < 0 || qs >= g.Q) {
                set_error(a.ctl, ERR_CONSIST, 10);
                qs = 0;
            }
            int i, j;
            frame_to_global(b, g.axis, g.r, qs, i, j);
            const Acc c = cell_cost<KIND, DIM>(pd, i, j, a.d);
            if constexpr (KIND == KIND_ABS) {
                total_i = rr.end_i;
                if (b.known_i >= 0 && b.known_i != total_i) set_error(a.ctl, ERR_CONSIST, 11);
                known_l = out[qs];
                known_r = total_i - known_l + c;
            } else {
                total_f = rr.end_f;
                kl_f = out[qs];
                kr_f = total_f - kl_f + c;
            }
        }
    } else {
        // F + B - C over the split row (Lemma 2); argmin, ties to the lowest column
        const Sweep& fw = a.sweeps[2 * bi];
        const Sweep& bw = a.sweeps[2 * bi + 1];
        const Acc* F = static_cast<const Acc*>(a.outpool) + fw.out_off;
        const Acc* B = static_cast<const Acc*>(a.outpool) + bw.out_off;
        double best_f = __longlong_as_double(0x7ff0000000000000LL);
        long long best_i = LLONG_MAX;
        int best_q = INT_MAX;
        for (int q = threadIdx.x; q < g.Q; q += blockDim.x) {
            int i, j;
            frame_to_global(b, g.axis, g.r, q, i, j);
            const Acc c = cell_cost<KIND, DIM>(pd, i, j, a.d);
            if constexpr (KIND == KIND_ABS) {
                const long long S = (long long)F[q] + (long long)B[q] - (long long)c;
                if (S < best_i) {
                    best_i = S;
                    best_q = q;
                }
            } else {
                const double S = F[q] + B[q] - c;
                if (S < best_f) {
                    best_f = S;
                    best_q = q;
                }
            }
        }
        // block argmin (value, then lowest column)
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const double of = __shfl_down_sync(kFull, best_f, o);
            const long long oi = __shfl_down_sync(kFull, best_i, o);
            const int oq = __shfl_down_sync(kFull, best_q, o);
            const bool take = (KIND == KIND_ABS) ? (oi < best_i || (oi == best_i && oq < best_q))
                                                 : (of < best_f || (of == best_f && oq < best_q));
            if (take) {
                best_f = of;
                best_i = oi;
                best_q = oq;
            }
        }
        if (lane == 0) {
            s_val[wid] = best_f;
            s_ival[wid] = best_i;
            s_q[wid] = best_q;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
                const bool take = (KIND == KIND_ABS)
                                      ? (s_ival[w] < best_i || (s_ival[w] == best_i && s_q[w] < best_q))
                                      : (s_val[w] < best_f || (s_val[w] == best_f && s_q[w] < best_q));
                if (take) {
                    best_f = s_val[w];
                    best_i = s_ival[w];
                    best_q = s_q[w];
                }
            }
            qs = best_q;
            if constexpr (KIND == KIND_ABS) {
                total_i = best_i;
                if (b.known_i >= 0 && b.known_i != total_i) set_error(a.ctl, ERR_CONSIST, 12);
                known_l = F[qs];
                known_r = B[qs];
            } else {
                total_f = best_f;
                kl_f = F[qs];
                kr_f = B[qs];
            }
        }
    }
    if (threadIdx.x == 0) {
        if (b.flags & BOX_ROOT) {
            a.pres[b.pair].cost_i = total_i;
            a.pres[b.pair].cost_f = total_f;
        }
        Box L = b, Rb = b;
        L.flags = 0;
        Rb.flags = 0;
        if (g.axis == 0) {
            L.H = g.r + 1;
            L.W = qs + 1;
            Rb.i0 = b.i0 + g.r;
            Rb.j0 = b.j0 + qs;
            Rb.H = b.H - g.r;
            Rb.W = b.W - qs;
        } else {
            L.H = qs + 1;
            L.W = g.r + 1;
            Rb.i0 = b.i0 + qs;
            Rb.j0 = b.j0 + g.r;
            Rb.H = b.H - qs;
            Rb.W = b.W - g.r;
        }
        L.known_i = known_l;
        Rb.known_i = known_r;
        L.known_f = kl_f;
        Rb.known_f = kr_f;
        emit_child(a, L);
        emit_child(a, Rb);
    }
}

template <int KIND, int DIM>
__global__ void __launch_bounds__(256) split_kernel(SplitArgs a) {
    // after a planning or sweep error the sweep outputs are not valid
    if (ld_relaxed(&a.ctl->err) != ERR_NONE) return;
    for (int bi = blockIdx.x; bi < a.n_boxes; bi += gridDim.x) {
        split_box<KIND, DIM>(a, bi);
        __syncthreads();
    }
}

cudaError_t launch_split(const SplitArgs& a, cudaStream_t st) {
    if (a.n_boxes <= 0) return cudaSuccess;
    const int grid = a.n_boxes < 65535 ? a.n_boxes : 65535;
    if (a.kind == KIND_ABS) split_kernel<KIND_ABS, 1><<<grid, 256, 0, st>>>(a);
    else if (a.d == 12) split_kernel<KIND_EUC, 12><<<grid, 256, 0, st>>>(a);
    else split_kernel<KIND_EUC, 0><<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- base case

// Shared memory per warp: 2-bit backpointers of up to kBaseAreaMax cells
// (rows are the shorter side, 16 pointers per word, each row word-aligned) and
// the boundary row between consecutive 32-row bands.
constexpr int kPtrWords = (int)(kBaseAreaMax / 16) + 182;  // P*ceil(Q/16) <= A/16 + sqrt(A)
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
    for (int bi = blockIdx.x * kBaseWarps + w; bi < a.n_base; bi += gridDim.x * kBaseWarps) {
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
                Acc up = __shfl_up_sync(kFull, cur, 1);
                const bool act = rowok && q >= 0 && q < Q;
                if (lane == 0) up = (band == 0 || !act) ? INF : row[q];
                if (act) {
                    Frame<KIND, DIM> yc;
                    yc.load(cs, cbase + q, a.d);
                    const Acc c = frame_cost(xr, yc);
                    const Acc m = min3(dprev, up, left);
                    uint32_t pt;
                    if (p == 0 && q == 0) pt = 3;
                    else if (dprev == m) pt = 0;
                    else if (vf) pt = (up == m) ? 1 : 2;
                    else pt = (left == m) ? 2 : 1;
                    cur = m + c;
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
            const Acc t = __shfl_down_sync(kFull, end_v, o);
            end_v = min(end_v, t);
        }
        if (lane == 0) {
            if constexpr (KIND == KIND_ABS) {
                if (b.known_i >= 0 && b.known_i != (long long)end_v) set_error(a.ctl, ERR_CONSIST, 20);
                if (b.flags & BOX_ROOT) a.pres[b.pair].cost_i = end_v;
            } else {
                if (b.flags & BOX_ROOT) a.pres[b.pair].cost_f = end_v;
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
    int grid = (a.n_base + kBaseWarps - 1) / kBaseWarps;
    if (grid > 65535) grid = 65535;
    base_kernel<KIND, DIM><<<grid, 32 * kBaseWarps, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_base(const BaseArgs& a, cudaStream_t st) {
    if (a.n_base <= 0) return cudaSuccess;
    if (a.kind == KIND_ABS) return launch_base_t<KIND_ABS, 1>(a, st);
    if (a.d == 12) return launch_base_t<KIND_EUC, 12>(a, st);
    return launch_base_t<KIND_EUC, 0>(a, st);
}

// ---------------------------------------------------------------- path assembly

// One block per pair: lengths of the per-row column runs, their exclusive scan
// (the row offsets in the path) and the structural checks of a warping path.
__global__ void __launch_bounds__(1024) assemble_scan_kernel(AssembleArgs a) {
    __shared__ long long carry;
    const int pb = blockIdx.x;
    const PairDesc pd = a.pairs[pb];
    const int32_t* jlo = a.jlo + pd.row_off;
    const int32_t* jhi = a.jhi + pd.row_off;
    int32_t* off = a.off + pd.row_off;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < pd.M; base += blockDim.x) {
        const int i = base + threadIdx.x;
        long long len = 0;
        if (i < pd.M) {
            const int lo = jlo[i], hi = jhi[i];
            bool ok = lo <= hi && lo >= 0 && hi < pd.N;
            if (i == 0) ok = ok && lo == 0;
            else ok = ok && (lo == jhi[i - 1] || lo == jhi[i - 1] + 1);
            if (i == pd.M - 1) ok = ok && hi == pd.N - 1;
            if (!ok) set_error(a.ctl, ERR_PATH, i);
            len = ok ? hi - lo + 1 : 0;
        }
        long long tot;
        const long long e = block_excl_scan(len, &tot);
        if (i < pd.M) off[i] = (int32_t)(carry + e);
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) a.pres[pb].K = (int32_t)carry;
}

__global__ void assemble_scatter_kernel(AssembleArgs a) {
    const int pb = blockIdx.y;
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

// Exactness guard of the int32 accumulator: every accumulated cost is at most
// max|x - y| * (M + N - 1), which must stay below 2^29.
__global__ void int_range_kernel(const PairDesc* pairs, int n_pairs, LevelCtl* ctl) {
    __shared__ int smin[2], smax[2];
    for (int pb = blockIdx.x; pb < n_pairs; pb += gridDim.x) {
        const PairDesc pd = pairs[pb];
        if (threadIdx.x < 2) {
            smin[threadIdx.x] = INT_MAX;
            smax[threadIdx.x] = INT_MIN;
        }
        __syncthreads();
        int mn[2] = {INT_MAX, INT_MAX}, mx[2] = {INT_MIN, INT_MIN};
        for (int i = threadIdx.x; i < pd.M; i += blockDim.x) {
            const int v = static_cast<const int32_t*>(pd.X)[i];
            mn[0] = min(mn[0], v);
            mx[0] = max(mx[0], v);
        }
        for (int j = threadIdx.x; j < pd.N; j += blockDim.x) {
            const int v = static_cast<const int32_t*>(pd.Y)[j];
            mn[1] = min(mn[1], v);
            mx[1] = max(mx[1], v);
        }
        for (int t = 0; t < 2; ++t) {
            atomicMin(&smin[t], mn[t]);
            atomicMax(&smax[t], mx[t]);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const long long c1 = (long long)smax[0] - smin[1], c2 = (long long)smax[1] - smin[0];
            const long long cmax = c1 > c2 ? c1 : c2;
            if (cmax * ((long long)pd.M + pd.N - 1) >= (1LL << 29)) set_error(ctl, ERR_OVERFLOW, pb);
        }
        __syncthreads();
    }
}

cudaError_t launch_int_range_check(const PairDesc* pairs, int n_pairs, LevelCtl* ctl, cudaStream_t st) {
    int g = n_pairs < 1024 ? n_pairs : 1024;
    int_range_kernel<<<g, 256, 0, st>>>(pairs, n_pairs, ctl);
    return cudaGetLastError();
}

}  // namespace dtwb
