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
// Band hand-off.  The band's last row goes to a global boundary row as 64-bit
// words that carry the writing band's epoch (dtw_common.cuh), two per column.  A
// reader accepts a word only when it bears the epoch of the band above, so no
// fence, flag or reset is needed and stale words from earlier bands, levels or
// calls are rejected.  Lane 0 of the band below keeps a ring of upcoming blocks
// in shared memory, filled PF blocks ahead with cp.async: in steady state the
// block it needs is already on the SM.  When a prefetched block turns out
// stale (the band above was not yet there), lane 0 reads it directly until it
// is valid and then re-synchronises: it waits until the band above is LEAD
// blocks ahead and refills the ring.
//
// Scheduling.  The kernel is persistent: each warp takes band tickets from an
// atomic counter until the level's bands are exhausted.  Tickets are issued in
// sweep order and, inside a sweep, top band first, so the band a warp waits on
// always belongs to a warp that is already running: no deadlock, whatever the
// grid size.  Every wait is bounded; on expiry the kernel records ERR_TIMEOUT
// and the band finishes on garbage, which the host turns into DTW_ETIMEOUT.
//
// Split tags (integer kind, canonical pivot fallback).  In a tag sweep, the
// cells of frame row tag_row carry their own column as tag, and every later
// cell copies the tag of its backpointer (first minimum in the order DIAG, UP,
// LEFT).  The tag reaching the last cell names the column where the canonical
// backtrace meets the split row, so that cell lies on the canonical path.
#include "dtw_common.cuh"
#include "dtw_kernels.h"

namespace dtwb {

namespace {

constexpr int kWarpsPerBlock = 4;
constexpr int PF = 16;         // prefetch distance, in column blocks
constexpr int RING = 64;       // ring slots per warp (> 31 + PF: lanes read Y up to 31 blocks back)
constexpr int LEAD = PF + 8;   // lead of the band above required after a re-sync

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void st_words2(unsigned long long* p, unsigned long long a, unsigned long long b) {
    asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ unsigned long long mkword(uint32_t payload, uint32_t epoch) {
    return ((unsigned long long)epoch << 32) | payload;
}

// Polls one boundary word until it bears epoch ep (bounded).  Returns the word;
// on expiry records ERR_TIMEOUT and returns a word with a different epoch.
__device__ __noinline__ unsigned long long wait_word(const unsigned long long* p, uint32_t ep, LevelCtl* ctl,
                                                     int spin_limit, int band) {
    unsigned long long w = 0;
    int it = 0;
    for (;; ++it) {
        w = ld_word(p);
        if (word_epoch(w) == ep) break;
        if (it >= spin_limit || ((it & 63) == 63 && ld_relaxed(&ctl->err) != ERR_NONE)) {
            set_error(ctl, ERR_TIMEOUT, band);
            break;
        }
        __nanosleep(32);
    }
    atomicAdd(&ctl->polls, (unsigned long long)it);
    return w;
}

// Bytes of one frame's features in the Y part of a ring slot.
template <int KIND, int DIM>
struct YBytes {
    static constexpr int v = KIND == KIND_ABS ? 4 : 4 * DIM;
};

}  // namespace

// Ring slot of a warp: [boundary words of one column block][Y frames of the block].
template <int KIND, int U, int DIM, int NWMAX>
struct Slot {
    static constexpr int BWMAX = U * NWMAX;                       // boundary words
    static constexpr int YOFF = BWMAX * 8;                         // byte offset of the Y frames
    static constexpr int YB = U * YBytes<KIND, DIM>::v;            // Y bytes (0 when DIM == 0)
    static constexpr int BYTES = YOFF + ((YB + 15) & ~15);
};

// TAGM: 0 untagged rows, 1 every row of the band tagged, 2 the band holds tag_row.
// VF:   the vertical frame move (p-1, q) precedes the horizontal one (p, q-1)
//       in the backpointer order (true when frame rows run along X).
// NW:   boundary words per column (1: integer value; 2: value and tag, or the
//       two halves of a double).
// SPECIAL: the band holds an out row or the sweep's last row.
template <int KIND, int R, int U, int DIM, int NWMAX, int NW, int TAGM, bool VF, bool SPECIAL>
__device__ __noinline__ void run_band(const Sweep& S, int sweep_idx, int band, bool publisher, const SweepArgs& A,
                                      unsigned char* ring) {
    using Acc = typename AccOf<KIND>::T;
    using SL = Slot<KIND, U, DIM, NWMAX>;
    constexpr bool TAG = TAGM != 0;
    constexpr bool YRING = DIM > 0;  // Y frames travel through the ring (fixed dimension)
    constexpr int BW = U * NW;       // boundary words per block
    static_assert(BW % 2 == 0, "boundary blocks are written as 16-byte pairs");
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

    unsigned long long* buf = A.bufpool + S.buf_off;
    Acc* outp = static_cast<Acc*>(A.outpool) + S.out_off;
    const int out_row0 = S.out_row0, nout = S.nout;
    const int end_k = S.rows - 1 - p0;
    const int tag_row = S.tag_row;
    const int Q = S.Q, nblk = S.nblk, rev = S.dir;
    const long long cbase = S.cbase;
    const int cstep = S.cstep;
    const char* colbytes = static_cast<const char*>(S.colseq);
    constexpr int FB = YBytes<KIND, DIM>::v;  // bytes per frame
    const uint32_t ep_in = S.epoch0 + (uint32_t)band;  // epoch of the band above
    const uint32_t ep_out = ep_in + 1u;
    const bool has_above = band > 0;
    Acc end_v = INF;
    int end_t = -1;
    bool need_sync = true, gave_up = false;
    const int nsteps = nblk + 31;

    // lane 0: copies of column block b (boundary words from the band above, Y frames)
    auto issue = [&](int b) {
        unsigned char* slot = ring + (b & (RING - 1)) * SL::BYTES;
        if (has_above) {
            const unsigned long long* src = buf + (size_t)b * BW;
#pragma unroll
            for (int i = 0; i < BW / 2; ++i) cp_async16(slot + 16 * i, src + 2 * i);
        }
        if constexpr (YRING) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = min(b * U + u, Q - 1);
                const char* src = colbytes + (cbase + (long long)cstep * q) * FB;
                if constexpr (FB == 4) {
                    cp_async4(slot + SL::YOFF + 4 * u, src);
                } else {
#pragma unroll
                    for (int e = 0; e < FB / 16; ++e) cp_async16(slot + SL::YOFF + FB * u + 16 * e, src + 16 * e);
                }
            }
        }
    };

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
            if (need_sync) {
                cp_async_wait<0>();  // no older copy may land in the ring after the refill
                if (has_above && !gave_up) {
                    const int tb = min(cb + LEAD, nblk - 1);
                    const unsigned long long w =
                        wait_word(buf + (size_t)tb * BW + BW - 1, ep_in, A.ctl, A.spin_limit, band);
                    if (word_epoch(w) != ep_in) gave_up = true;
                    atomicAdd(&A.ctl->resyncs, 1ULL);
                }
#pragma unroll 1
                for (int i = 0; i < PF; ++i) {
                    if (cb + i < nblk) issue(cb + i);
                    cp_async_commit();
                }
                need_sync = false;
            }
            if (cb + PF < nblk) issue(cb + PF);
            cp_async_commit();
            cp_async_wait<PF>();  // the copies of block cb have landed
            if (!has_above || gave_up) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    upv[u] = INF;
                    upt[u] = 0;
                }
            } else {
                const unsigned long long* sl =
                    reinterpret_cast<const unsigned long long*>(ring + (cb & (RING - 1)) * SL::BYTES);
                unsigned long long w[BW];
                bool ok = true;
#pragma unroll
                for (int i = 0; i < BW; ++i) {
                    w[i] = sl[i];
                    ok = ok && word_epoch(w[i]) == ep_in;
                }
                if (!ok) {  // copied before the band above wrote it: read it directly, then re-sync
#pragma unroll
                    for (int i = 0; i < BW; ++i) {
                        if (!gave_up && word_epoch(w[i]) != ep_in) {
                            w[i] = wait_word(buf + (size_t)cb * BW + i, ep_in, A.ctl, A.spin_limit, band);
                            if (word_epoch(w[i]) != ep_in) gave_up = true;
                        }
                    }
                    need_sync = true;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if constexpr (NW == 1) {
                        upv[u] = (Acc)(int32_t)word_payload(w[u]);
                        upt[u] = 0;
                    } else if constexpr (KIND == KIND_ABS) {
                        upv[u] = (Acc)(int32_t)word_payload(w[2 * u]);
                        upt[u] = (int32_t)word_payload(w[2 * u + 1]);
                    } else {
                        upv[u] = (Acc)__hiloint2double((int)word_payload(w[2 * u + 1]), (int)word_payload(w[2 * u]));
                        upt[u] = 0;
                    }
                }
            }
        }
        __syncwarp();  // lane 0's completed copies are visible to the whole warp
        if (active) {
            Frame<KIND, DIM> yc[U];
            if constexpr (YRING) {
                const unsigned char* ys = ring + (cb & (RING - 1)) * SL::BYTES + SL::YOFF;
#pragma unroll
                for (int u = 0; u < U; ++u) yc[u].load_shared(ys + FB * u);
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int q = min(cb * U + u, Q - 1);
                    yc[u].load(S.colseq, cbase + (long long)cstep * q, A.d);
                }
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
        if (publisher && lane == 31 && active) {
            unsigned long long w[BW];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if constexpr (NW == 1) {
                    w[u] = mkword((uint32_t)bot[u], ep_out);
                } else if constexpr (KIND == KIND_ABS) {
                    w[2 * u] = mkword((uint32_t)bot[u], ep_out);
                    w[2 * u + 1] = mkword((uint32_t)bott[u], ep_out);
                } else {
                    w[2 * u] = mkword((uint32_t)__double2loint((double)bot[u]), ep_out);
                    w[2 * u + 1] = mkword((uint32_t)__double2hiint((double)bot[u]), ep_out);
                }
            }
            unsigned long long* dst = buf + (size_t)cb * BW;
#pragma unroll
            for (int i = 0; i < BW / 2; ++i) st_words2(dst + 2 * i, w[2 * i], w[2 * i + 1]);
        }
    }
    if (lane == 0) cp_async_wait<0>();
    __syncwarp();
    if constexpr (SPECIAL) {
        if (end_k >= 0 && end_k < R) {
            SweepRes* r = A.res + sweep_idx;
            if constexpr (KIND == KIND_ABS) r->end_i = end_v;
            else r->end_f = end_v;
            r->end_tag = end_t;
        }
    }
}

template <int KIND, int R, int U, int DIM, int NWMAX, int NW, int TAGM, bool VF>
__device__ __forceinline__ void run_band_s(const Sweep& S, int si, int band, bool pub, const SweepArgs& A,
                                           unsigned char* ring, bool special) {
    if (special) run_band<KIND, R, U, DIM, NWMAX, NW, TAGM, VF, true>(S, si, band, pub, A, ring);
    else run_band<KIND, R, U, DIM, NWMAX, NW, TAGM, VF, false>(S, si, band, pub, A, ring);
}

// TAGS: the launch may contain tagged sweeps (integer kind), whose boundary
// rows carry two words per column; untagged integer sweeps use one.
template <int KIND, int R, int U, int DIM, bool TAGS>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) sweep_kernel(SweepArgs A) {
    constexpr int NWMAX = (KIND == KIND_EUC || TAGS) ? 2 : 1;
    using SL = Slot<KIND, U, DIM, NWMAX>;
    __shared__ __align__(16) unsigned char s_ring[kWarpsPerBlock][RING * SL::BYTES];
    const int lane = threadIdx.x & 31;
    unsigned char* ring = s_ring[threadIdx.x >> 5];
    const int n_sweeps = A.ctl->n_sweeps;
    const long long n_tickets = A.ctl->n_tickets;
    for (;;) {
        long long t = 0;
        if (lane == 0) t = (long long)atomicAdd(&A.ctl->ticket, 1ULL);
        t = __shfl_sync(kFull, t, 0);
        if (t >= n_tickets) break;
        if (ld_relaxed(&A.ctl->err) != ERR_NONE) break;
        // the sweep owning ticket t: last sweep whose band_begin <= t (empty
        // sweeps share their successor's band_begin and are skipped)
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
        const bool special = (S.nout > 0 && S.out_row0 < b_hi && S.out_row0 + S.nout > b_lo) || (S.rows - 1 < b_hi);
        if constexpr (KIND == KIND_EUC) {
            run_band_s<KIND, R, U, DIM, NWMAX, 2, 0, true>(S, lo, band, publisher, A, ring, special);
        } else if (!TAGS || S.tag_row < 0) {
            run_band_s<KIND, R, U, DIM, NWMAX, 1, 0, true>(S, lo, band, publisher, A, ring, special);
        } else if constexpr (TAGS) {
            const bool vf = S.axis == 0;
            if (b_hi <= S.tag_row) {
                run_band_s<KIND, R, U, DIM, NWMAX, 2, 0, true>(S, lo, band, publisher, A, ring, special);
            } else if (b_lo > S.tag_row) {
                if (vf) run_band_s<KIND, R, U, DIM, NWMAX, 2, 1, true>(S, lo, band, publisher, A, ring, special);
                else run_band_s<KIND, R, U, DIM, NWMAX, 2, 1, false>(S, lo, band, publisher, A, ring, special);
            } else {
                if (vf) run_band_s<KIND, R, U, DIM, NWMAX, 2, 2, true>(S, lo, band, publisher, A, ring, special);
                else run_band_s<KIND, R, U, DIM, NWMAX, 2, 2, false>(S, lo, band, publisher, A, ring, special);
            }
        }
    }
}

// ---------------------------------------------------------------- launchers

template <int KIND, int R, int U, int DIM, bool TAGS>
static cudaError_t launch_one(const SweepArgs& A, int num_sms, cudaStream_t st) {
    static int nb = 0;
    if (nb == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<KIND, R, U, DIM, TAGS>,
                                                      32 * kWarpsPerBlock, 0);
        if (nb < 1) nb = 1;
    }
    sweep_kernel<KIND, R, U, DIM, TAGS><<<num_sms * nb, 32 * kWarpsPerBlock, 0, st>>>(A);
    return cudaGetLastError();
}

// Variants: integer |x-y| (R=2, U=4, tagged rows allowed) and Euclidean d=12
// (R=2, U=2) or any other d read from memory (R=2, U=2).
int sweep_block_cols(int kind, int d) { return kind == KIND_ABS ? 4 : 2; }
int sweep_band_rows(int kind, int d) { return 64; }

cudaError_t launch_sweep(int kind, int d, bool tags, const SweepArgs& A, int num_sms, cudaStream_t st) {
    if (kind == KIND_ABS) {
        if (tags) return launch_one<KIND_ABS, 2, 4, 1, true>(A, num_sms, st);
        return launch_one<KIND_ABS, 2, 4, 1, false>(A, num_sms, st);
    }
    if (d == 12) return launch_one<KIND_EUC, 2, 2, 12, false>(A, num_sms, st);
    return launch_one<KIND_EUC, 2, 2, 0, false>(A, num_sms, st);
}

}  // namespace dtwb
