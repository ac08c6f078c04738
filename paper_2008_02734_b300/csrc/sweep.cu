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
// warp shuffle.  Nothing but one boundary row per sweep, the split rows and the
// last cell's value leaves the SM: the D matrix itself is never stored (linear
// memory, Section 3.2).
//
// Strips.  A thread block has kG compute warps and one loader warp.  It takes
// tickets of kG consecutive bands of the level (band numbering runs through
// the level's sweeps in order, top band first), so a block usually holds kG
// adjacent bands of one sweep, or several short sweeps side by side.  Warp g
// hands its band's last row to warp g+1 through a ring of column blocks in
// shared memory, published with release/acquire progress counters: the
// hand-off costs one shared store per step on the producer side and one shared
// load on the consumer side, and lanes other than lane 0 / lane 31 take no
// part.  Only the last warp of a block writes to global memory: a boundary row
// of 64-bit words that carry the writing band's epoch (dtw_common.cuh).  The
// block that owns the band below reads that row with its loader warp, which
// polls 32 columns at a time until every word bears the expected epoch and
// copies the payloads into the first warp's ring.  No fence, flag or reset is
// needed in global memory: stale words from earlier bands, levels or calls
// carry other epochs and are not accepted.
//
// Scheduling.  The kernel is persistent.  Tickets are issued in band order, so
// the band a warp waits on belongs to the same block or to a block that took an
// earlier ticket and is already running: no deadlock, whatever the grid.  Every
// wait is bounded; on expiry the kernel records ERR_TIMEOUT, the waiting warp
// finishes on garbage, and the host turns it into DTW_ETIMEOUT.
//
// Split tags (integer kind, canonical pivot fallback).  In a tag sweep, the
// cells of frame row tag_row carry their own column as tag, and every later
// cell copies the tag of its backpointer (first minimum in the order DIAG, UP,
// LEFT).  The tag reaching the last cell names the column where the canonical
// backtrace meets the split row, so that cell lies on the canonical path.
#include "dtw_common.cuh"
#include "dtw_kernels.h"

// Lane block of the integer sweep (rows x columns per lane and step).
#ifndef DTW_INT_R
#define DTW_INT_R 4
#endif
#ifndef DTW_INT_U
#define DTW_INT_U 4
#endif

namespace dtwb {

namespace {

constexpr int kG = 4;                  // compute warps (bands) per block
constexpr int kThreads = 32 * (kG + 1);  // + the loader warp
constexpr int RS = 64;                 // ring slots (column blocks) per warp boundary
constexpr int KP = 8;                  // progress counters are published every KP blocks
constexpr int kQuickPolls = 8;         // polls before a waiting warp starts to sleep

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ int ld_acquire_cta(const int* p) {
    int v;
    asm volatile("ld.acquire.cta.shared.b32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta(int* p, int v) {
    asm volatile("st.release.cta.shared.b32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void st_words2(unsigned long long* p, unsigned long long a, unsigned long long b) {
    asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ unsigned long long mkword(uint32_t payload, uint32_t epoch) {
    return ((unsigned long long)epoch << 32) | payload;
}
__device__ __forceinline__ void prefetch_l1(const void* p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Stores / loads n 32-bit words at a shared address aligned to 4*n bytes (n <= 4)
// or to 16 bytes (n a multiple of 4).
template <int N>
__device__ __forceinline__ void st_shared_words(uint32_t* p, const uint32_t* w) {
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int i = 0; i < N; i += 4)
            *reinterpret_cast<uint4*>(p + i) = make_uint4(w[i], w[i + 1], w[i + 2], w[i + 3]);
    } else if constexpr (N % 2 == 0) {
#pragma unroll
        for (int i = 0; i < N; i += 2) *reinterpret_cast<uint2*>(p + i) = make_uint2(w[i], w[i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) p[i] = w[i];
    }
}
template <int N>
__device__ __forceinline__ void ld_shared_words(const uint32_t* p, uint32_t* w) {
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int i = 0; i < N; i += 4) {
            const uint4 t = *reinterpret_cast<const uint4*>(p + i);
            w[i] = t.x;
            w[i + 1] = t.y;
            w[i + 2] = t.z;
            w[i + 3] = t.w;
        }
    } else if constexpr (N % 2 == 0) {
#pragma unroll
        for (int i = 0; i < N; i += 2) {
            const uint2 t = *reinterpret_cast<const uint2*>(p + i);
            w[i] = t.x;
            w[i + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) w[i] = p[i];
    }
}

// Per-warp wait statistics, flushed once per band.
struct WaitStats {
    unsigned long long waits = 0, polls = 0;
};

// Spins until *ctr >= target (a shared progress counter; warp-uniform call).
// Bounded: on expiry records ERR_TIMEOUT and returns the last value seen.
__device__ __forceinline__ int wait_counter(const int* ctr, int target, LevelCtl* ctl, int spin_limit, int info,
                                            bool& gave_up, WaitStats& ws) {
    int v = ld_acquire_cta(ctr);
    if (v >= target || gave_up) return v;
    ++ws.waits;
    for (int it = 1;; ++it) {
        if (it >= spin_limit || ((it & 63) == 0 && ld_relaxed(&ctl->err) != ERR_NONE)) {
            set_error(ctl, ERR_TIMEOUT, info);
            gave_up = true;
            return v;
        }
        if (it > kQuickPolls) __nanosleep(32);
        v = ld_acquire_cta(ctr);
        ++ws.polls;
        if (v >= target) return v;
    }
}

// Payload words of one column in rings and boundary rows.
template <int KIND, int NW>
__device__ __forceinline__ void pack(typename AccOf<KIND>::T v, int t, uint32_t* w) {
    if constexpr (KIND == KIND_ABS) {
        w[0] = (uint32_t)v;
        if constexpr (NW == 2) w[1] = (uint32_t)t;
    } else {
        w[0] = (uint32_t)__double2loint((double)v);
        w[1] = (uint32_t)__double2hiint((double)v);
    }
}
template <int KIND, int NW>
__device__ __forceinline__ void unpack(const uint32_t* w, typename AccOf<KIND>::T& v, int& t) {
    if constexpr (KIND == KIND_ABS) {
        v = (int32_t)w[0];
        t = NW == 2 ? (int)w[1] : 0;
    } else {
        v = __hiloint2double((int)w[1], (int)w[0]);
        t = 0;
    }
}

}  // namespace

// Shared memory of a block: one ring per compute warp (ring g feeds warp g; the
// loader writes ring 0, warp g-1 writes ring g).
template <int U, int NWMAX>
struct StripSmem {
    static constexpr int SLOT = U * NWMAX;  // words per ring slot
    __align__(16) uint32_t ring[kG][RS * SLOT];
    int prog[kG];  // column blocks written into ring g
    int cons[kG];  // column blocks consumed from ring g
    long long ticket;
    int stop;
};

// Where a band's last row goes.
constexpr int OUT_NONE = 0;    // last band of its sweep
constexpr int OUT_RING = 1;    // to the next warp of the block
constexpr int OUT_GLOBAL = 2;  // to the block holding the band below (boundary row in global memory)

// One band.  TAGM: 0 untagged rows, 1 every row of the band tagged, 2 the band
// holds tag_row.  VF: the vertical frame move (p-1, q) precedes the horizontal
// one (p, q-1) in the backpointer order (true when frame rows run along X).
// NW: payload words per column (1: integer value; 2: value and tag, or the two
// halves of a double).  SPECIAL: the band holds an out row or the sweep's last row.
template <int KIND, int R, int U, int DIM, int NWMAX, int NW, int TAGM, bool VF, bool SPECIAL>
__device__ __noinline__ void run_band(const Sweep* __restrict__ sp, int sweep_idx, int band, int out_mode,
                                      const SweepArgs& A, uint32_t* rin, int* prog_in, int* cons_in, uint32_t* rout,
                                      int* prog_out, const int* cons_out) {
    using Acc = typename AccOf<KIND>::T;
    constexpr bool TAG = TAGM != 0;
    constexpr int SLOT = U * NWMAX;  // ring slot stride (words)
    constexpr int BW = U * NW;       // payload words per block
    static_assert(BW % 2 == 0, "boundary blocks are written as 16-byte pairs");
    const int lane = threadIdx.x & 31;
    const Acc INF = AccOf<KIND>::inf();

    const int rows = sp->rows, Q = sp->Q, nblk = sp->nblk, rev = sp->dir;
    const int rbase = sp->rbase, rstep = sp->rstep;
    const long long cbase = sp->cbase;
    const int cstep = sp->cstep;
    const void* rowseq = sp->rowseq;
    const void* colseq = sp->colseq;
    const int out_row0 = sp->out_row0, nout = sp->nout, tag_row = sp->tag_row;
    const uint32_t ep_out = sp->epoch0 + (uint32_t)band + 1u;
    unsigned long long* buf = A.bufpool + sp->buf_off;
    Acc* outp = static_cast<Acc*>(A.outpool) + sp->out_off;
    const int p0 = band * (32 * R) + lane * R;
    const int end_k = rows - 1 - p0;

    Frame<KIND, DIM> xr[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int p = min(p0 + k, rows - 1);
        xr[k].load(rowseq, (long long)rbase + (long long)rstep * p, A.d);
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

    // column frames of the lane's next block (lane l starts at block -l: clamped)
    auto load_cols = [&](Frame<KIND, DIM>* y, int cb) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = min(max(cb * U + u, 0), Q - 1);
            y[u].load(colseq, cbase + (long long)cstep * q, A.d);
        }
    };
    Frame<KIND, DIM> yn[U];
    load_cols(yn, -lane);

    const long long fbytes = KIND == KIND_ABS ? 4 : 4LL * (DIM > 0 ? DIM : A.d);  // bytes per column frame
    const bool has_above = band > 0;
    Acc end_v = INF;
    int end_t = -1;
    bool gave_up = false;
    WaitStats ws;
    int avail = 0;  // blocks known to be in rin
    int room = RS;  // blocks that may be written to rout
    const int nsteps = nblk + 31;
    for (int s = 0; s < nsteps; ++s) {
        const int cb = s - lane;
        const bool active = cb >= 0 && cb < nblk;
        Frame<KIND, DIM> yc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) yc[u] = yn[u];
        if (lane == 0 && s + 16 < nblk) {
            const int q = min((s + 16) * U, Q - 1);
            prefetch_l1(static_cast<const char*>(colseq) + (cbase + (long long)cstep * q) * fbytes);
        }
        load_cols(yn, cb + 1);

        Acc upv[U];
        int upt[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            upv[u] = __shfl_up_sync(kFull, bot[u], 1);
            if constexpr (TAG) upt[u] = __shfl_up_sync(kFull, bott[u], 1);
            else upt[u] = 0;
        }
        // lane 0: the band above's last row over block s
        if (has_above) {
            if (s < nblk && s >= avail) avail = wait_counter(prog_in, s + 1, A.ctl, A.spin_limit, band, gave_up, ws);
            if (lane == 0 && s < nblk) {
                uint32_t w[BW];
                ld_shared_words<BW>(rin + (s % RS) * SLOT, w);
#pragma unroll
                for (int u = 0; u < U; ++u) unpack<KIND, NW>(w + u * NW, upv[u], upt[u]);
            }
            if (lane == 0 && s < nblk && ((s + 1) % KP == 0 || s == nblk - 1)) st_release_cta(cons_in, s + 1);
        } else if (lane == 0) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                upv[u] = INF;
                upt[u] = 0;
            }
        }

        if (active) {
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
                        const int orow = p0 + k - out_row0;
                        if ((unsigned)orow < (unsigned)nout && q < Q)
                            outp[(size_t)(rev ? nout - 1 - orow : orow) * Q + (rev ? Q - 1 - q : q)] = nv;
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

        // lane 31: the band's last row over block s-31, for the band below
        const int ob = s - 31;
        if (out_mode == OUT_RING && ob >= 0) {
            if (ob >= room) room = wait_counter(cons_out, ob + 1 - RS, A.ctl, A.spin_limit, band, gave_up, ws) + RS;
            if (lane == 31) {
                uint32_t w[BW];
#pragma unroll
                for (int u = 0; u < U; ++u) pack<KIND, NW>(bot[u], bott[u], w + u * NW);
                st_shared_words<BW>(rout + (ob % RS) * SLOT, w);
                if ((ob + 1) % KP == 0 || ob == nblk - 1) st_release_cta(prog_out, ob + 1);
            }
        } else if (out_mode == OUT_GLOBAL && ob >= 0 && lane == 31) {
            uint32_t w[BW];
#pragma unroll
            for (int u = 0; u < U; ++u) pack<KIND, NW>(bot[u], bott[u], w + u * NW);
            unsigned long long* dst = buf + (size_t)ob * BW;
#pragma unroll
            for (int i = 0; i < BW / 2; ++i) st_words2(dst + 2 * i, mkword(w[2 * i], ep_out), mkword(w[2 * i + 1], ep_out));
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
    if (lane == 0 && ws.waits) {
        atomicAdd(&A.ctl->resyncs, ws.waits);
        atomicAdd(&A.ctl->polls, ws.polls);
    }
}

// The loader warp: copies the boundary row written by the block above (global
// memory, epoch-stamped words) into ring 0, 32 columns per round.
template <int U, int NWMAX, int NW>
__device__ __noinline__ void run_loader(const Sweep* __restrict__ sp, int band, const SweepArgs& A, uint32_t* ring,
                                        int* prog, const int* cons) {
    constexpr int SLOT = U * NWMAX;
    static_assert(32 % U == 0, "a round of 32 columns covers whole blocks");
    const int lane = threadIdx.x & 31;
    const unsigned long long* buf = A.bufpool + sp->buf_off;
    const uint32_t ep = sp->epoch0 + (uint32_t)band;  // epoch of the band above
    const int nblk = sp->nblk;
    const int ncol = nblk * U;
    bool gave_up = false;
    WaitStats ws;
    int room = RS;
    for (int c0 = 0; c0 < ncol; c0 += 32) {
        const int b1 = min((c0 + 32) / U, nblk);
        if (b1 > room) room = wait_counter(cons, b1 - RS, A.ctl, A.spin_limit, band, gave_up, ws) + RS;
        const int col = c0 + lane;
        unsigned long long w[NW];
        bool ok = col >= ncol;
        for (int it = 0;; ++it) {
            if (!ok) {
#pragma unroll
                for (int i = 0; i < NW; ++i) w[i] = ld_word(buf + (size_t)col * NW + i);
                ok = true;
#pragma unroll
                for (int i = 0; i < NW; ++i) ok = ok && word_epoch(w[i]) == ep;
            }
            if (__all_sync(kFull, ok) || gave_up) break;
            if (it == 0) ++ws.waits;
            ++ws.polls;
            if (it >= A.spin_limit || ((it & 63) == 63 && ld_relaxed(&A.ctl->err) != ERR_NONE)) {
                set_error(A.ctl, ERR_TIMEOUT, band);
                gave_up = true;
                break;
            }
            __nanosleep(64);
        }
        if (col < ncol) {
            uint32_t* dst = ring + ((col / U) % RS) * SLOT + (col % U) * NW;
#pragma unroll
            for (int i = 0; i < NW; ++i) dst[i] = word_payload(w[i]);
        }
        __threadfence_block();
        __syncwarp();
        if (lane == 0) st_release_cta(prog, b1);
    }
    if (lane == 0 && ws.waits) {
        atomicAdd(&A.ctl->resyncs, ws.waits);
        atomicAdd(&A.ctl->polls, ws.polls);
    }
}

template <int KIND, int R, int U, int DIM, int NWMAX, int NW, int TAGM, bool VF>
__device__ __forceinline__ void run_band_s(bool special, const Sweep* sp, int si, int band, int om,
                                           const SweepArgs& A, uint32_t* rin, int* pin, int* cin, uint32_t* rout,
                                           int* pout, const int* cout) {
    if (special) run_band<KIND, R, U, DIM, NWMAX, NW, TAGM, VF, true>(sp, si, band, om, A, rin, pin, cin, rout, pout, cout);
    else run_band<KIND, R, U, DIM, NWMAX, NW, TAGM, VF, false>(sp, si, band, om, A, rin, pin, cin, rout, pout, cout);
}

// Index of the sweep holding level band gb: the last sweep whose band_begin is
// <= gb (empty sweeps share their successor's band_begin and are skipped).
__device__ __forceinline__ int find_sweep(const Sweep* sweeps, int n_sweeps, long long gb) {
    int lo = 0, hi = n_sweeps - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sweeps[mid].band_begin <= gb) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// TAGS: the launch may contain tagged sweeps (integer kind), whose rows carry
// two payload words per column; untagged integer sweeps use one.
template <int KIND, int R, int U, int DIM, bool TAGS>
__global__ void __launch_bounds__(kThreads) sweep_kernel(const __grid_constant__ SweepArgs A) {
    constexpr int NWMAX = (KIND == KIND_EUC || TAGS) ? 2 : 1;
    __shared__ StripSmem<U, NWMAX> sm;
    const int warp = threadIdx.x >> 5;
    const int n_sweeps = A.ctl->n_sweeps;
    const long long n_tickets = A.ctl->n_tickets;
    const long long n_bands = A.ctl->n_bands;
    for (;;) {
        if (threadIdx.x == 0) {
            sm.ticket = (long long)atomicAdd(&A.ctl->ticket, 1ULL);
            sm.stop = ld_relaxed(&A.ctl->err) != ERR_NONE;
        }
        if (threadIdx.x < kG) {
            sm.prog[threadIdx.x] = 0;
            sm.cons[threadIdx.x] = 0;
        }
        __syncthreads();
        const long long t = sm.ticket;
        if (t >= n_tickets || sm.stop) break;
        if (warp < kG) {
            const long long gb = t * kG + warp;
            if (gb < n_bands) {
                const int si = find_sweep(A.sweeps, n_sweeps, gb);
                const Sweep* sp = A.sweeps + si;
                const int band = (int)(gb - sp->band_begin);
                const int nbands = sp->nbands, rows = sp->rows, tag_row = sp->tag_row;
                int om = band + 1 < nbands ? (warp + 1 < kG ? OUT_RING : OUT_GLOBAL) : OUT_NONE;
                if (gb == A.skip_ticket) om = OUT_NONE;
                const int BR = 32 * R;
                const int b_lo = band * BR, b_hi = b_lo + BR;  // band rows [b_lo, b_hi)
                const bool special =
                    (sp->nout > 0 && sp->out_row0 < b_hi && sp->out_row0 + sp->nout > b_lo) || (rows - 1 < b_hi);
                uint32_t* rin = sm.ring[warp];
                int* pin = &sm.prog[warp];
                int* cin = &sm.cons[warp];
                const int wn = warp + 1 < kG ? warp + 1 : warp;  // unused when om != OUT_RING
                uint32_t* rout = sm.ring[wn];
                int* pout = &sm.prog[wn];
                const int* cout = &sm.cons[wn];
                if constexpr (KIND == KIND_EUC) {
                    run_band_s<KIND, R, U, DIM, NWMAX, 2, 0, true>(special, sp, si, band, om, A, rin, pin, cin, rout,
                                                                   pout, cout);
                } else if (!TAGS || tag_row < 0) {
                    run_band_s<KIND, R, U, DIM, NWMAX, 1, 0, true>(special, sp, si, band, om, A, rin, pin, cin, rout,
                                                                   pout, cout);
                } else if constexpr (TAGS) {
                    const bool vf = sp->axis == 0;
                    if (b_hi <= tag_row) {
                        run_band_s<KIND, R, U, DIM, NWMAX, 2, 0, true>(special, sp, si, band, om, A, rin, pin, cin,
                                                                       rout, pout, cout);
                    } else if (b_lo > tag_row) {
                        if (vf)
                            run_band_s<KIND, R, U, DIM, NWMAX, 2, 1, true>(special, sp, si, band, om, A, rin, pin, cin,
                                                                           rout, pout, cout);
                        else
                            run_band_s<KIND, R, U, DIM, NWMAX, 2, 1, false>(special, sp, si, band, om, A, rin, pin,
                                                                            cin, rout, pout, cout);
                    } else {
                        if (vf)
                            run_band_s<KIND, R, U, DIM, NWMAX, 2, 2, true>(special, sp, si, band, om, A, rin, pin, cin,
                                                                           rout, pout, cout);
                        else
                            run_band_s<KIND, R, U, DIM, NWMAX, 2, 2, false>(special, sp, si, band, om, A, rin, pin,
                                                                            cin, rout, pout, cout);
                    }
                }
            }
        } else {
            // the loader serves warp 0 when its band continues a band of an earlier block
            const long long gb = t * kG;
            if (gb < n_bands) {
                const int si = find_sweep(A.sweeps, n_sweeps, gb);
                const Sweep* sp = A.sweeps + si;
                const int band = (int)(gb - sp->band_begin);
                if (band > 0) {
                    if (KIND == KIND_EUC || (TAGS && sp->tag_row >= 0))
                        run_loader<U, NWMAX, 2>(sp, band, A, sm.ring[0], &sm.prog[0], &sm.cons[0]);
                    else
                        run_loader<U, NWMAX, 1>(sp, band, A, sm.ring[0], &sm.prog[0], &sm.cons[0]);
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- launchers

template <int KIND, int R, int U, int DIM, bool TAGS>
static cudaError_t launch_one(const SweepArgs& A, int num_sms, cudaStream_t st) {
    static int nb = 0;
    if (nb == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<KIND, R, U, DIM, TAGS>, kThreads, 0);
        if (nb < 1) nb = 1;
    }
    sweep_kernel<KIND, R, U, DIM, TAGS><<<num_sms * nb, kThreads, 0, st>>>(A);
    return cudaGetLastError();
}

// Variants: integer |x-y| with an R x U block per lane and step (tagged rows
// allowed or not), Euclidean d=12 (R=2, U=2) and any other d read from memory
// (R=2, U=2).  A lane's R x U block is a small wavefront of its own: its
// anti-diagonals give the scheduler independent cells, and the per-step
// hand-off work (shuffles, ring, boundary stores) is paid once per block.
constexpr int kIntR = DTW_INT_R, kIntU = DTW_INT_U;
int sweep_block_cols(int kind, int d) { return kind == KIND_ABS ? kIntU : 2; }
int sweep_band_rows(int kind, int d) { return kind == KIND_ABS ? 32 * kIntR : 64; }
int sweep_group_bands() { return kG; }

cudaError_t launch_sweep(int kind, int d, bool tags, const SweepArgs& A, int num_sms, cudaStream_t st) {
    if (kind == KIND_ABS) {
        if (tags) return launch_one<KIND_ABS, kIntR, kIntU, 1, true>(A, num_sms, st);
        return launch_one<KIND_ABS, kIntR, kIntU, 1, false>(A, num_sms, st);
    }
    if (d == 12) return launch_one<KIND_EUC, 2, 2, 12, false>(A, num_sms, st);
    return launch_one<KIND_EUC, 2, 2, 0, false>(A, num_sms, st);
}

}  // namespace dtwb
