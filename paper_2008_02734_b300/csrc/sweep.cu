// Tiled anti-diagonal wavefront sweep of the accumulated-cost recurrence
// (Section 2.1, Eq. "recurrence"; the diagonal order of Algorithm 1, Section 3.1).
//
// Work decomposition.  A sweep covers frame rows [0, rows) x frame columns
// [0, Q).  Its rows are cut into bands of 32*R rows; one warp owns one band and
// walks it left to right in blocks of U columns.  Lane l owns rows
// [l*R, l*R+R) of the band and, at step s, evaluates the R x U cells of column
// block s-l: the lanes of a warp hold 32 consecutive blocks of an anti-diagonal
// of blocks, so every dependency (UP, LEFT, DIAG) is either in the lane's own
// registers or was produced by the lane above one step earlier and arrives by
// warp shuffle.  The band's last row goes to a global boundary row (one entry
// per column, O(Q) per sweep) and a per-band progress counter is advanced with a
// release store every PUB blocks; the band below acquires it before reading.
// Nothing but that boundary row, the split row and the last cell's value leaves
// the SM: the D matrix itself is never stored (linear memory, Section 3.2).
//
// Scheduling.  The kernel is persistent: each warp takes band tickets from an
// atomic counter until the level's bands are exhausted.  Tickets are issued in
// sweep order and, inside a sweep, top band first, so the band a warp waits on
// always belongs to a warp that is already running: no deadlock, whatever the
// grid size.  Every wait is bounded; on expiry the kernel records ERR_TIMEOUT
// and the band finishes on garbage, which the host turns into DTW_ETIMEOUT.
//
// Split tags (integer kind, the canonical pivot).  In a tag sweep, the cells of
// frame row tag_row carry their own column as tag, and every later cell copies
// the tag of its backpointer (first minimum in the order DIAG, UP, LEFT).  The
// tag reaching the last cell names the column where the canonical backtrace
// meets the split row, so that cell lies on the canonical optimal path.
#include "dtw_common.cuh"
#include "dtw_kernels.h"

namespace dtwb {

// TAGM: 0 untagged rows, 1 every row of the band tagged, 2 the band holds tag_row.
// VF:   the vertical frame move (p-1, q) precedes the horizontal one (p, q-1)
//       in the backpointer order (true when frame rows run along X).
// SPECIAL: the band holds the out row or the sweep's last row.
template <int KIND, int R, int U, int DIM, int TAGM, bool VF, bool SPECIAL>
__device__ __noinline__ void run_band(const Sweep& S, int sweep_idx, int band, bool publisher,
                                      const SweepArgs& A) {
    using Acc = typename AccOf<KIND>::T;
    constexpr int PUB = 2;
    constexpr bool TAG = TAGM != 0;
    const int lane = threadIdx.x & 31;
    const Acc INF = AccOf<KIND>::inf();
    const int p0 = band * (32 * R) + lane * R;

    Frame<KIND, DIM> xr[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int p = min(p0 + k, S.rows - 1);
        xr[k].load(S.rowseq, (long long)S.rbase + (long long)S.rstep * p, A.d);
    }

    Acc L[R];  // D(p0+k, q-1): the column left of the current one
    int LT[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        L[k] = INF;
        LT[k] = 0;
    }
    // D(p0-1, q-1) for the lane's top row; the virtual corner D(-1,-1) = 0
    // starts the recurrence at (0,0) (Eq. "dtwboundary").
    Acc dprev = (p0 == 0) ? AccOf<KIND>::zero() : INF;
    int dprevt = 0;
    Acc bot[U];  // the lane's last row over the current block, for the lane below
    int bott[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        bot[u] = INF;
        bott[u] = 0;
    }

    Acc* rb = static_cast<Acc*>(A.bufpool) + S.buf_off;
    int* tb = A.tagpool + S.buf_off;
    int* prog = A.progpool + S.prog_off;
    Acc* outp = static_cast<Acc*>(A.outpool) + S.out_off;
    const int out_k = S.out_row - p0;
    const int end_k = S.rows - 1 - p0;
    const int tag_row = S.tag_row;
    const int Q = S.Q, nblk = S.nblk, rev = S.dir;
    const void* const colseq = S.colseq;
    const long long cbase = S.cbase, cstep = S.cstep;
    Acc end_v = INF;
    int end_t = -1;
    int seen = (band == 0) ? 0x7fffffff : 0;  // blocks of the band above known to be published
    const int nsteps = nblk + 31;

    for (int s = 0; s < nsteps; ++s) {
        const int cb = s - lane;
        const bool active = cb >= 0 && cb < nblk;
        Acc upv[U];
        int upt[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            upv[u] = __shfl_up_sync(kFull, bot[u], 1);
            if constexpr (TAG) upt[u] = __shfl_up_sync(kFull, bott[u], 1);
            else upt[u] = 0;
        }
        if (lane == 0 && active) {
            if (band == 0) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    upv[u] = INF;
                    upt[u] = 0;
                }
            } else {
                if (seen <= cb) {
                    int it = 0;
                    for (;;) {
                        seen = ld_acquire(prog + band - 1);
                        if (seen > cb) break;
                        if (++it > A.spin_limit || ld_relaxed(&A.ctl->err) != ERR_NONE) {
                            set_error(A.ctl, ERR_TIMEOUT, band);
                            seen = 0x7fffffff;  // finish the band on garbage
                            break;
                        }
                        __nanosleep(64);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    upv[u] = __ldcg(rb + cb * U + u);
                    if constexpr (TAG) upt[u] = __ldcg(tb + cb * U + u);
                }
            }
        }
        if (active) {
            Frame<KIND, DIM> yc[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = min(cb * U + u, Q - 1);
                yc[u].load(colseq, cbase + cstep * q, A.d);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = cb * U + u;
                Acc a_up = upv[u];
                int t_up = upt[u];
                Acc a_dg = (u == 0) ? dprev : upv[u - 1];
                int t_dg = (u == 0) ? dprevt : upt[u - 1];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const Acc c = frame_cost(xr[k], yc[u]);
                    const Acc lf = L[k];
                    const Acc m = min3(a_dg, a_up, lf);
                    const Acc nv = m + c;
                    int t = 0;
                    if constexpr (TAG) {
                        const int t_lf = LT[k];
                        // tag of the backpointer: first minimum among DIAG, UP, LEFT
                        if constexpr (VF) t = (a_dg == m) ? t_dg : ((a_up == m) ? t_up : t_lf);
                        else t = (a_dg == m) ? t_dg : ((lf == m) ? t_lf : t_up);
                        if constexpr (TAGM == 2) t = (p0 + k == tag_row) ? q : t;
                        t_dg = t_lf;
                        t_up = t;
                        LT[k] = t;
                    }
                    if constexpr (SPECIAL) {
                        if (k == out_k && q < Q) outp[rev ? Q - 1 - q : q] = nv;
                        if (k == end_k && q == Q - 1) {
                            end_v = nv;
                            end_t = t;
                        }
                    }
                    a_dg = lf;
                    a_up = nv;
                    L[k] = nv;
                }
                bot[u] = a_up;
                bott[u] = t_up;
            }
            dprev = upv[U - 1];
            dprevt = upt[U - 1];
        }
        if (publisher && lane == 31 && active) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                rb[cb * U + u] = bot[u];
                if constexpr (TAG) tb[cb * U + u] = bott[u];
            }
            if ((cb + 1) % PUB == 0 || cb == nblk - 1) st_release(prog + band, cb + 1);
        }
    }
    if constexpr (SPECIAL) {
        if (end_k >= 0 && end_k < R) {
            SweepRes* r = A.res + sweep_idx;
            if constexpr (KIND == KIND_ABS) r->end_i = end_v;
            else r->end_f = end_v;
            r->end_tag = end_t;
        }
    }
}

template <int KIND, int R, int U, int DIM, int TAGM, bool VF>
__device__ __forceinline__ void run_band_s(const Sweep& S, int si, int band, bool pub, const SweepArgs& A,
                                           bool special) {
    if (special) run_band<KIND, R, U, DIM, TAGM, VF, true>(S, si, band, pub, A);
    else run_band<KIND, R, U, DIM, TAGM, VF, false>(S, si, band, pub, A);
}

template <int KIND, int R, int U, int DIM, bool TAGS>
__global__ void __launch_bounds__(128) sweep_kernel(SweepArgs A) {
    const int lane = threadIdx.x & 31;
    const int n_sweeps = A.ctl->n_sweeps;
    const long long n_tickets = A.ctl->n_tickets;
    for (;;) {
        long long t = 0;
        if (lane == 0) t = (long long)atomicAdd(&A.ctl->ticket, 1ULL);
        t = __shfl_sync(kFull, t, 0);
        if (t >= n_tickets) break;
        if (ld_relaxed(&A.ctl->err) != ERR_NONE) break;
        // the sweep owning ticket t: last sweep whose band_begin <= t
        int lo = 0, hi = n_sweeps - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (A.sweeps[mid].band_begin <= t) lo = mid;
            else hi = mid - 1;
        }
        const Sweep S = A.sweeps[lo];
        const int band = (int)(t - S.band_begin);
        const int BR = 32 * R;
        const int b_lo = band * BR, b_hi = b_lo + BR;  // band rows [b_lo, b_hi)
        const bool publisher = band < S.nbands - 1 && t != A.skip_ticket;
        const bool special = (S.out_row >= b_lo && S.out_row < b_hi) || (S.rows - 1 < b_hi);
        if (!TAGS || S.tag_row < 0 || b_hi <= S.tag_row) {
            run_band_s<KIND, R, U, DIM, 0, true>(S, lo, band, publisher, A, special);
        } else {
            const bool vf = S.axis == 0;
            if (b_lo > S.tag_row) {
                if (vf) run_band_s<KIND, R, U, DIM, 1, true>(S, lo, band, publisher, A, special);
                else run_band_s<KIND, R, U, DIM, 1, false>(S, lo, band, publisher, A, special);
            } else {
                if (vf) run_band_s<KIND, R, U, DIM, 2, true>(S, lo, band, publisher, A, special);
                else run_band_s<KIND, R, U, DIM, 2, false>(S, lo, band, publisher, A, special);
            }
        }
    }
}

// ---------------------------------------------------------------- launchers

template <int KIND, int R, int U, int DIM, bool TAGS>
static cudaError_t launch_one(const SweepArgs& A, int grid, cudaStream_t st) {
    sweep_kernel<KIND, R, U, DIM, TAGS><<<grid, 128, 0, st>>>(A);
    return cudaGetLastError();
}

template <int KIND, int R, int U, int DIM, bool TAGS>
static int occupancy_blocks() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<KIND, R, U, DIM, TAGS>, 128, 0);
    return nb > 0 ? nb : 1;
}

// Variants: integer |x-y| (R=2, U=4; tagged or not) and Euclidean d=12
// (R=2, U=2) or any other d read from memory (R=2, U=2).
int sweep_block_cols(int kind, int d) { return kind == KIND_ABS ? 4 : 2; }
int sweep_band_rows(int kind, int d) { return 64; }

cudaError_t launch_sweep(int kind, int d, bool tags, const SweepArgs& A, int num_sms, cudaStream_t st) {
    if (kind == KIND_ABS) {
        if (tags) {
            static int nb = occupancy_blocks<KIND_ABS, 2, 4, 1, true>();
            return launch_one<KIND_ABS, 2, 4, 1, true>(A, num_sms * nb, st);
        }
        static int nb = occupancy_blocks<KIND_ABS, 2, 4, 1, false>();
        return launch_one<KIND_ABS, 2, 4, 1, false>(A, num_sms * nb, st);
    }
    if (d == 12) {
        static int nb = occupancy_blocks<KIND_EUC, 2, 2, 12, false>();
        return launch_one<KIND_EUC, 2, 2, 12, false>(A, num_sms * nb, st);
    }
    static int nb = occupancy_blocks<KIND_EUC, 2, 2, 0, false>();
    return launch_one<KIND_EUC, 2, 2, 0, false>(A, num_sms * nb, st);
}

}  // namespace dtwb
