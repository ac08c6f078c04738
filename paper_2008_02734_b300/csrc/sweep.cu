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
// Strips.  A thread block has G compute warps and one loader warp.  It takes
// tickets, each a group of G consecutive bands of one sweep: group j of a
// sweep is bands jG .. jG+G-1.  The plan writes the ticket map in group-major
// order (every sweep's group 0, then every sweep's group 1, ...); without a map
// (a sweep of 1024 groups or more) tickets are G consecutive bands of the
// level's band numbering, which may put short sweeps side by side.  Warp g
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
// Scheduling.  The kernel is persistent.  In both orders the band a warp waits
// on (the band above, of the same sweep) belongs to the same block or to an
// earlier ticket, whose block is already running: no deadlock, whatever the
// grid.  Every
// wait is bounded; on expiry the kernel records ERR_TIMEOUT, the waiting warp
// finishes on garbage, and the host turns it into DTW_ETIMEOUT.
//
// Split tags (integer kind, canonical pivot fallback).  In a tag sweep, the
// cells of frame row tag_row carry their own column as tag, and every later
// cell copies the tag of its backpointer (first minimum in the order DIAG, UP,
// LEFT).  The tag reaching the last cell names the column where the canonical
// backtrace meets the split row, so that cell lies on the canonical path.
#include <atomic>
#include <climits>
#include <type_traits>

#include "dtw_common.cuh"
#include "dtw_kernels.h"
#include "split.cuh"

// Lane block of the integer sweep (rows x columns per lane and step).
#ifndef DTW_INT_R
#define DTW_INT_R 4
#endif
#ifndef DTW_INT_U
#define DTW_INT_U 4
#endif
// Lane block of the Euclidean d=12 sweep.
#ifndef DTW_EUC_R
#define DTW_EUC_R 2
#endif
#ifndef DTW_EUC_U
#define DTW_EUC_U 2
#endif

namespace dtwb {

namespace {

// Compute warps (bands) per block, G: integer kind 2, Euclidean kinds 4.  An
// integer step is short, so a level's few bands do better spread over more
// SMs; the longer Euclidean steps gain from four warps sharing a frame stream.
#ifndef DTW_SWEEP_G_INT
#define DTW_SWEEP_G_INT 2
#endif
#ifndef DTW_SWEEP_G_EUC
#define DTW_SWEEP_G_EUC 4
#endif
// The BF16 tensor-core form's block always holds four bands: the M = 128 rows of
// one MMA.
constexpr int kGEucB = 4;
template <int KIND>
__host__ __device__ constexpr int group_of() {
    return int_kind(KIND) ? DTW_SWEEP_G_INT : (KIND == KIND_EUCB ? kGEucB : DTW_SWEEP_G_EUC);
}
template <int KIND>
__host__ __device__ constexpr int threads_of() {
    // + the loader warp; the BF16 tensor-core form adds its tile warp
    return 32 * (group_of<KIND>() + 1 + (KIND == KIND_EUCB ? 1 : 0));
}
// Resident blocks per SM of the throughput form of the d = 12 Euclidean sweep:
// the register cap that lets this many blocks share an SM (96 registers a
// thread for four 160-thread blocks, against the compiler's 128 and three).
#ifndef DTW_EUC_MINB
#define DTW_EUC_MINB 4
#endif
constexpr int kEucMinB = DTW_EUC_MINB;
constexpr int kGMax = 8;  // the frame ring partition covers up to 8 warps
constexpr int URS = 64;                  // slots (column blocks) of a row ring
#ifndef DTW_SWEEP_KC
#define DTW_SWEEP_KC 8
#endif
#ifndef DTW_SWEEP_UNROLL
#define DTW_SWEEP_UNROLL 4
#endif
#ifndef DTW_SWEEP_UNROLL_EUC
#define DTW_SWEEP_UNROLL_EUC 0
#endif
// The block's last band warp hands its last row to the loader warp through one
// more shared-memory ring, and the loader writes it to the global boundary row
// (1), instead of storing the epoch-stamped words itself every step (0).
#ifndef DTW_LOADER_DRAIN
#define DTW_LOADER_DRAIN 1
#endif
#ifndef DTW_EUC_YPREFETCH
#define DTW_EUC_YPREFETCH 0
#endif
constexpr int KC = DTW_SWEEP_KC;         // steps per group: rings are synchronised once per group
// Drained by the loader: every kind but the integer kind's fully unrolled
// variant, whose steady 8-step groups publish one row ring per group and whose
// cross-block hand-off then lags by up to a group (integer pair 2.35 ms with
// the band's own stores against 2.52 with the drain; the others gain 2-6%).
template <int KIND, bool FULL>
__host__ __device__ constexpr bool drain_of() { return DTW_LOADER_DRAIN != 0 && !(int_kind(KIND) && FULL); }
// Integer kinds: steps per loop iteration of a steady group; the local
// alignment's sweeps (KIND_LOCAL, with the floor and the best-node tracking)
// take 2 (their two passes 5.98 -> 5.71 ms on the 20000 x 24000 workload with
// 2 for every integer kind, where the integer pair and edit distance lose 10%).
template <int KIND>
__host__ __device__ constexpr int int_unroll() { return KIND == KIND_LOCAL ? 2 : DTW_SWEEP_UNROLL; }
// Euclidean kinds (longer steps, larger code): steps per loop iteration of a
// steady group, by kind and dimension.  Measured (chroma pair 2000 x 2500, the
// 256-pair chroma batch, the 60000 x 75000 d=64 pair): d=12 with 2 steps 1.46 ms
// and 94.1 ms against 1.54 and 95.4 with 1; the d=64 FP32-cost form with 4
// steps 114.5 ms against 117.1 (with 2: 127.9); the BF16 form and the
// compensated d=64 form unchanged.  DTW_SWEEP_UNROLL_EUC > 0 sets one factor
// for every Euclidean variant.
template <int KIND, int DIM>
__host__ __device__ constexpr int euc_unroll() {
    return DTW_SWEEP_UNROLL_EUC > 0 ? DTW_SWEEP_UNROLL_EUC : (DIM == 12 ? 2 : (DIM == 64 && KIND == KIND_EUC ? 4 : 1));
}

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
// The same store, executed only where pred holds (a predicated instruction, so
// that the hot loop carries no divergent branch around it).
__device__ __forceinline__ void st_words2_if(bool pred, unsigned long long* p, unsigned long long a,
                                             unsigned long long b) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\t@q st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};\n\t}" ::"l"(p),
        "l"(a), "l"(b), "r"((int)pred)
        : "memory");
}
// A relaxed store of a progress counter, executed only where pred holds; after a
// fence.acq_rel.cta of the storing thread it publishes like a release.
__device__ __forceinline__ void st_relaxed_cta_if(bool pred, int* p, int v) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q st.relaxed.cta.shared.b32 [%0], %1;\n\t}" ::"r"(
                     smem_addr(p)),
                 "r"(v), "r"((int)pred)
                 : "memory");
}
__device__ __forceinline__ unsigned long long mkword(uint32_t payload, uint32_t epoch) {
    return ((unsigned long long)epoch << 32) | payload;
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
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
// The same store, executed only where pred holds (predicated instructions for
// whole 16-byte units).
template <int N>
__device__ __forceinline__ void st_shared_words_if(bool pred, uint32_t* p, const uint32_t* w) {
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int i = 0; i < N; i += 4)
            asm volatile(
                "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %5, 0;\n\t@q st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n\t}" ::"r"(
                    smem_addr(p + i)),
                "r"(w[i]), "r"(w[i + 1]), "r"(w[i + 2]), "r"(w[i + 3]), "r"((int)pred)
                : "memory");
    } else {
        if (pred) st_shared_words<N>(p, w);
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

// Stores one 16-byte chunk of out-row accumulators (out_chunk of them), only
// where pred holds: a predicated instruction, so that a step with out rows in
// some of its lanes carries no divergent branch.
template <typename T>
__device__ __forceinline__ void store_chunk_if(bool pred, T* p, const T* v) {
    static_assert(sizeof(T) * out_chunk<T>() == 16, "16-byte chunks");
    uint32_t w[4];
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = (uint32_t)v[i];
    } else if constexpr (std::is_same<T, double>::value) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            w[2 * i] = (uint32_t)__double2loint(v[i]);
            w[2 * i + 1] = (uint32_t)__double2hiint(v[i]);
        }
    } else {  // DF: hi, lo
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            w[2 * i] = __float_as_uint(v[i].hi);
            w[2 * i + 1] = __float_as_uint(v[i].lo);
        }
    }
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %5, 0;\n\t@q st.global.v4.b32 [%0], {%1, %2, %3, %4};\n\t}" ::"l"(p),
                 "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"((int)pred)
                 : "memory");
}

// Per-warp wait statistics, flushed once per band.
struct WaitStats {
    unsigned long long waits = 0, polls = 0;
};

// Spins until *ctr >= target (a shared progress counter; warp-uniform call).
// The writer is another warp of the same block, on another scheduler, so the
// wait spins without sleeping.  Bounded: on expiry records ERR_TIMEOUT and
// returns the last value seen.
__device__ __forceinline__ int wait_counter(const int* ctr, int target, LevelCtl* ctl, int spin_limit, int info,
                                            bool& gave_up, WaitStats& ws) {
    int v = ld_acquire_cta(ctr);
    if (v >= target || gave_up) return v;
    ++ws.waits;
    for (int it = 1;; ++it) {
        if (it >= spin_limit || ((it & 255) == 0 && ld_relaxed(&ctl->err) != ERR_NONE)) {
            set_error(ctl, ERR_TIMEOUT, info);
            gave_up = true;
            return v;
        }
        v = ld_acquire_cta(ctr);
        ++ws.polls;
        if (v >= target) return v;
    }
}

// Payload words of one column in rings and boundary rows.
template <int KIND, int NW>
__device__ __forceinline__ void pack(typename AccOf<KIND>::T v, int t, uint32_t* w) {
    if constexpr (int_kind(KIND)) {
        w[0] = (uint32_t)v;
        if constexpr (NW == 2) w[1] = (uint32_t)t;
    } else if constexpr (std::is_same<typename AccOf<KIND>::T, DF>::value) {
        w[0] = __float_as_uint(v.hi);
        w[1] = __float_as_uint(v.lo);
    } else {
        w[0] = (uint32_t)__double2loint((double)v);
        w[1] = (uint32_t)__double2hiint((double)v);
    }
}
template <int KIND, int NW>
__device__ __forceinline__ void unpack(const uint32_t* w, typename AccOf<KIND>::T& v, int& t) {
    if constexpr (int_kind(KIND)) {
        v = (int32_t)w[0];
        t = NW == 2 ? (int)w[1] : 0;
    } else if constexpr (std::is_same<typename AccOf<KIND>::T, DF>::value) {
        v = DF{__uint_as_float(w[0]), __uint_as_float(w[1])};
        t = 0;
    } else {
        v = __hiloint2double((int)w[1], (int)w[0]);
        t = 0;
    }
}

}  // namespace

// 32-bit words of one column frame in a frame ring (0: frames are read from
// global memory by every lane, the runtime-dimension variant).
template <int KIND, int DIM>
struct FrameWords {
    static constexpr int v = int_kind(KIND) ? 1 : (KIND == KIND_EUCB ? 0 : DIM);
};

// ---- BF16 tensor-core cost tiles (tcgen05, TMEM accumulators)
//
// A block of the BF16 form holds four bands of 32 rows of one sweep: 128 frame
// rows, the M = 128 of one tcgen05.mma.  The band warps write their rows' frames
// (BF16) into operand A once per ticket.  The bands run about 40 steps apart
// (the band below waits for the lanes of the band above), so each band has its
// own stream of 32-column tiles: for band g's tile t, a tile warp converts the
// 32 column frames into the band's operand B, takes their FP32 squared norms,
// and one of its threads issues four MMAs (K = 16 each, d = 64) into the band's
// TMEM slot and commits them to the slot's mbarrier.  TMEM lane i holds frame
// row i of the block, so band warp g (warp g % 4 reads lanes 32g..32g+31) loads
// its own rows' dot products with one tcgen05.ld (the other lanes of its slot go
// unused), forms the expanded cost and writes its ring of three 32 x 32 cost
// tiles in shared memory, which its skewed lanes read.  Each band has two slots
// (TMEM columns, operand B and norms): the tile warp fills one while the band
// works from the other.
constexpr int kTcBands = 4;
constexpr int kTcSlots = 2;                // per band
constexpr int kTcRows = 128;               // M: four bands of 32 frame rows
constexpr int kTcCols = 32;                // N: column frames per tile
constexpr int kTcK = 64;                   // K: the feature dimension
constexpr uint32_t kTcTmemCols = kTcBands * kTcSlots * kTcCols;  // 256 (a power of two >= 32)
// Operands in the no-swizzle K-major layout: 8-row x 16-byte core matrices;
// element (r, k) at (k / 8) * LBO + (r / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.
constexpr uint32_t kTcSBO = 128;                      // next 8 rows
constexpr uint32_t kTcLboA = (kTcRows / 8) * 128;     // next 8 k of A (2048 B)
constexpr uint32_t kTcLboB = (kTcCols / 8) * 128;     // next 8 k of B (512 B)
constexpr int kTcBytesA = kTcRows * kTcK * 2;
constexpr int kTcBytesB = kTcCols * kTcK * 2;

struct TcShared {
    __align__(128) unsigned char a[kTcBytesA];
    __align__(128) unsigned char b[kTcBands][kTcSlots][kTcBytesB];
    float yy[kTcBands][kTcSlots][kTcCols];        // squared norms of the tile's column frames
    // per band: three cost tiles, rows padded to 36 floats (16-byte rows; a step's
    // 8-byte read of two columns by the skewed lanes is conflict-free per half warp)
    __align__(16) float tile[kTcBands][3][32][36];
    unsigned long long mbar[kTcBands][kTcSlots];   // MMA completion per slot
    int produced[kTcBands];                        // per band: tiles whose MMAs are issued (running count)
    int consumed[kTcBands];                        // per band: tiles loaded from TMEM (running count)
    int tbase[kTcBands];                           // per band: running count at this ticket's start
    int a_ready[kTcBands];                         // ticket + 1 once the band warp's rows of operand A are written
    uint32_t tmem;                                 // TMEM base address of the block's slots
};

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 t = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&t);
}
__device__ __forceinline__ uint32_t tc_off(int r, int k, uint32_t lbo) {
    return (uint32_t)(k >> 3) * lbo + (uint32_t)(r >> 3) * kTcSBO + (uint32_t)(r & 7) * 16 + (uint32_t)(k & 7) * 2;
}
// Writes the 64 features of frame row r of an operand (BF16, 16 bytes at a time).
__device__ __forceinline__ void tc_store_row(unsigned char* base, int r, uint32_t lbo, const float* v) {
#pragma unroll
    for (int k8 = 0; k8 < kTcK / 8; ++k8) {
        const uint4 q = make_uint4(pack_bf16x2(v[8 * k8], v[8 * k8 + 1]), pack_bf16x2(v[8 * k8 + 2], v[8 * k8 + 3]),
                                   pack_bf16x2(v[8 * k8 + 4], v[8 * k8 + 5]), pack_bf16x2(v[8 * k8 + 6], v[8 * k8 + 7]));
        *reinterpret_cast<uint4*>(base + tc_off(r, 8 * k8, lbo)) = q;
    }
}
// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// Instruction descriptor of kind::f16: FP32 accumulators, BF16 A and B, both
// K-major, N = 32, M = 128.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcCols >> 3) << 17) |
                              ((uint32_t)(kTcRows >> 4) << 24);

// The BF16 form's cost from the TMEM dot product: sqrt(max(0, |x|^2 + |y|^2 -
// 2 x.y)) in FP32 (the square root rounded to nearest, or, with
// DTW_TC_SQRT_APPROX, the hardware approximation within 2 ulp: the form's error
// is set by the BF16 frames, some 2^-8 relative; default: the approximation).
#ifndef DTW_TC_SQRT_APPROX
#define DTW_TC_SQRT_APPROX 1
#endif
__device__ __forceinline__ float tc_cost(float xx, float yy, float dot) {
#if DTW_TC_SQRT_APPROX
    const float t = fmaxf(__fmaf_rn(-2.f, dot, __fadd_rn(xx, yy)), 0.f);
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(t));
    return r;
#else
    return expanded_cost(xx, yy, dot);
#endif
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(unsigned long long* m) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(m)) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* m, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
    return done != 0;
}
// D[tmem] (+)= A(desc) B(desc)^T, one thread.
__device__ __forceinline__ void tc_mma(uint32_t dt, uint64_t ad, uint64_t bd, bool acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(kTcIdesc), "r"((int)acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned long long* m) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(m))
                 : "memory");
}
// 32 consecutive TMEM columns of the warp's 32 lanes: lane l gets row l's values.
__device__ __forceinline__ void tc_ld32(uint32_t ta, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(ta)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Shared memory of a block.  Row ring g carries the last row of the band above
// warp g's band (written by warp g-1, or by the loader from global memory for
// warp 0); frame ring g carries the column frames of warp g's sweep (written by
// the loader).  Counters: blocks written (prog) and blocks released by the
// reader (cons).
//
// Warps of a block that belong to the same sweep read one frame stream: the
// ring of the first of them (ystream[g]).  The frame region of kYSlotsOf(G) column
// blocks is split among the block's streams when the block takes a ticket.  A
// stream read by w warps gets yslots(G, w) slots: a reader lags the warp above it
// by at most 40 steps when it waits on it, so the stream's first reader is at
// most 40(w-1) blocks ahead of its last one, which keeps 31 blocks (its lanes)
// plus a group in use; the loader's next round (chunk(w) blocks) must fit
// beside all that, otherwise the first reader could wait on the loader, the
// loader on the last reader and the last reader, through the chain of row
// rings, on the first one.  w = 5..8: 512 slots, rounds of 32; w = 4 or 3:
// 256, 32; w = 2: 128, 32; w = 1: 64, 16.  Every partition of four warps fits
// in 320 slots, every partition of eight in 1024.  That is the least room that
// cannot deadlock; a lower band that runs late (its waits on the band above
// make it lag by some 50 steps rather than 40) then holds back the first
// reader.  With two warps per block (the integer kind, 16-byte slots) the
// region is 512 slots and a stream gets 512 (two readers) or 256 (one); with two
// warps or fewer and large slots (more than 256 bytes) the least room applies:
// 128 slots, a stream 128 (two readers) or 64 (one).  Four warps with large
// slots (the d = 64 FP32-cost kinds, 528-byte slots) can also run with a tight
// ring: every ticket holds bands of one sweep only (the plan pads each sweep's
// bands to whole groups), so the one stream gets the least room of four
// readers, 40 x 3 + 31 + 8 + 32 = 191 blocks, as 192 slots (101 KB instead of
// 169: two blocks per SM instead of one).  The launch picks the ring: the
// tight one leaves out the end of the region (the ring is the last member of
// the block's shared memory).
constexpr int kYTight = 192;
__host__ __device__ constexpr bool ytight_capable(int G, bool big) { return big && G > 2 && G <= 4; }
__host__ __device__ constexpr int kYSlotsOf(int G, bool big = false) {
    return G > 4 ? 1024 : (G > 2 ? 320 : (big ? 128 : 512));
}
__host__ __device__ constexpr int yslots(int G, int w, bool big = false, bool tight = false) {
    return (tight && ytight_capable(G, big))
               ? kYTight
               : ((G <= 2 && !big) ? (w >= 2 ? 512 : 256) : (w >= 5 ? 512 : (w >= 3 ? 256 : (w == 2 ? 128 : 64))));
}
__host__ __device__ constexpr int ychunk(int w) { return w >= 2 ? 32 : 16; }

// A frame ring slot holds the U column frames of one block; lanes read the
// slots of consecutive blocks, so the slot stride is padded to an odd number of
// 16-byte units: the eight lanes of a 16-byte shared load then fall in eight
// different bank groups.
template <int U, int YW>
struct FrameSlot {
    static constexpr int W = (U * YW) % 4 != 0 || ((U * YW) / 4) % 2 == 1 ? U * YW : U * YW + 4;
};

template <int U, int NWMAX, int YW, int G>
struct StripSmem {
    static_assert(G >= 1 && G <= kGMax, "compute warps per block");
    static constexpr int YSW = FrameSlot<U, YW>::W;  // words per frame ring slot
    __align__(16) uint32_t uring[G + 1][URS * U * NWMAX];  // ring G: the last warp's row, for the loader
    static constexpr bool kBigSlot = YSW > 64;
    int uprog[G + 1], ucons[G + 1], yprog[G], ycons[G];
    int ybase[G], yrs[G], ychb[G];  // per stream: first slot, slots, blocks per loader round
    int sweep_of[G], band_of[G], ystream[G];
    long long ticket;
    int stop;
    int ntiles;  // BF16 tensor-core form: tiles of this ticket's sweep
    // last: a launch with the tight ring allocates only its first kYTight slots
    __align__(16) uint32_t yring[YW > 0 ? kYSlotsOf(G, kBigSlot) * YSW : 4];
};

// Column frame held by a lane: in registers, or (large fixed dimensions) a
// pointer into the frame ring.
template <int KIND, int DIM>
struct ColFrame {
    using T = Frame<KIND, DIM>;
};
template <>
struct ColFrame<KIND_EUC, 64> {
    using T = FrameRef<64>;
};
template <>
struct ColFrame<KIND_EUCF, 64> {
    using T = FrameRef<64>;
};

// One band.  TAGM: 0 untagged rows, 1 every row of the band tagged, 2 the band
// holds tag_row.  VF: the vertical frame move (p-1, q) precedes the horizontal
// one (p, q-1) in the backpointer order (true when frame rows run along X).
// NW: payload words per column (1: integer value; 2: value and tag, or the two
// halves of a double).  SPECIAL: the band holds an out row or the sweep's last row.
// to_ring / to_global: the band's last row goes to warp g+1 / to the block
// holding the next band (neither for the last band of a sweep).
//
// The step loop runs in groups of KC steps.  All waiting and publishing happens
// once per group, in warp-uniform code at the group's start; inside a group a
// step only reads the two rings (its inputs were loaded one step earlier),
// shuffles, evaluates its R x U cells and lets lane 31 store its last row.
// Groups in which every lane has a block (the band's steady state) run without
// per-lane activity tests.
template <int KIND, int R, int U, int DIM, int NWMAX, int NW, int TAGM, bool VF, bool SPECIAL, bool FULL>
__device__ __noinline__ void run_band(const Sweep* __restrict__ sp, int sweep_idx, int band, bool to_ring,
                                      bool to_global, const SweepArgs& A, StripSmem<U, NWMAX, FrameWords<KIND, DIM>::v, group_of<KIND>()>& sm,
                                      int g, TcShared* tc) {
    using Acc = typename AccOf<KIND>::T;
    using SM = StripSmem<U, NWMAX, FrameWords<KIND, DIM>::v, group_of<KIND>()>;
    constexpr int YW = FrameWords<KIND, DIM>::v;
    // BF16 tensor-core form: one row per lane, 16 column blocks of 2 per tile
    constexpr bool TC = KIND == KIND_EUCB;
    constexpr bool kDr = drain_of<KIND, FULL>();
    static_assert(!TC || (DIM == 64 && R == 1 && U == 2), "the tensor-core form is built for d = 64, R = 1, U = 2");
    constexpr bool TAG = TAGM != 0;
    constexpr int SLOT = U * NWMAX;  // row ring slot stride (words)
    constexpr int BW = U * NW;       // payload words per block
    static_assert(BW % 2 == 0, "boundary blocks are written as 16-byte pairs");
    const int lane = threadIdx.x & 31;
    const Acc INF = AccOf<KIND>::inf();

    const int rows = sp->rows, Q = sp->Q, nblk = sp->nblk;
    const int rbase = sp->rbase, rstep = sp->rstep;
    const void* rowseq = sp->rowseq;
    const int nout = sp->nout, tag_row = sp->tag_row;
    const int32_t esub = sp->esub, egap = sp->egap, ematch = sp->ematch;  // edit kinds
    const bool lfloor = sp->floor != 0;                                      // KIND_LOCAL
    const uint32_t ep_out = sp->epoch0 + (uint32_t)band + 1u;
    unsigned long long* buf = A.bufpool + sp->buf_off;
    Acc* outp = static_cast<Acc*>(A.outpool) + sp->out_off;
    const int p0 = band * (32 * R) + lane * R;
    const int end_k = rows - 1 - p0;
    const int end_u = (Q - 1) % U;  // the last cell's column within the last block
    // the last cell is read back only by cost sweeps (no out rows) and tag sweeps;
    // the half sweeps of an aligned box hand their last row over as out rows
    const bool need_end = nout == 0 || tag_row >= 0;
    const bool has_above = band > 0;
    // out rows of this lane: its rows meet one window of split rows at most
    // (windows are more than R rows apart), so valid row k is out row mo0 + k; in
    // the out-row layout (out_index) the lane's rows of column block cb start at
    // element mo0 * OC + cb * U * nout, row k OC further each
    constexpr int OC = out_chunk<Acc>();
    static_assert(U % OC == 0, "a lane's column block covers whole out-row chunks");
    static_assert(R <= kWinGap, "a lane's rows must not reach two windows of split rows");
    int mo0 = 0;
    bool ovalid[R];
#pragma unroll
    for (int k = R - 1; k >= 0; --k) {
        const int m = SPECIAL ? out_row_of(*sp, p0 + k) : -1;
        ovalid[k] = m >= 0;
        if (m >= 0) mo0 = m - k;
    }

    uint32_t* rin = sm.uring[g];
    constexpr int kG = group_of<KIND>();
    uint32_t* rout = sm.uring[kDr || g + 1 < kG ? g + 1 : g];
    const int ys = sm.ystream[g];
    constexpr int YSW = SM::YSW;
    const uint32_t* yr = sm.yring + (size_t)sm.ybase[ys] * YSW;
    const int ymask = sm.yrs[ys] - 1;
    // the frame ring slot of column block cb (cb >= -31); a tight ring is not a
    // power of two
    const bool tight = ytight_capable(group_of<KIND>(), SM::kBigSlot) && A.ytight != 0;
    auto yslot = [&](int cb) -> int { return tight ? (int)((unsigned)(cb + kYTight) % (unsigned)kYTight) : (cb & ymask); };
    if (!has_above) {
        // the row above the sweep: D(-1, q) = infinity (Eq. "dtwboundary")
        uint32_t w[NW];
        pack<KIND, NW>(INF, 0, w);
        for (int i = lane; i < URS * U; i += 32) {
#pragma unroll
            for (int k = 0; k < NW; ++k) rin[(i / U) * SLOT + (i % U) * NW + k] = w[k];
        }
        __syncwarp();
    }

    Frame<KIND, DIM> xr[R];
    if constexpr (!TC) {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int p = min(p0 + k, rows - 1);
            xr[k].load(rowseq, (long long)rbase + (long long)rstep * p, A.d);
        }
    }

    // ---- tensor-core cost tiles (BF16 form)
    // The lane's row frame goes into operand A (row 32g + lane) and its FP32
    // squared norm stays in a register.  Tile t (columns 32t .. 32t+31) is needed
    // when lane 0 reaches it; the band warp then waits for the tile warp's MMA of
    // it, loads its 32 lanes' dot products from TMEM and writes the costs of the
    // expanded form into its ring of three tiles (lane l reads only row l).
    float xxr = 0.f;
    if constexpr (TC) {
        Frame<KIND_EUC, 64> xf;
        xf.load(rowseq, (long long)rbase + (long long)rstep * min(p0, rows - 1), 64);
        xxr = sqnorm<64>(xf.v);
        tc_store_row(tc->a, 32 * g + lane, kTcLboA, xf.v);
        fence_proxy_async();  // the MMAs read operand A through the async proxy
        __syncwarp();
        if (lane == 0) st_release_cta(&tc->a_ready[g], (int)sm.ticket + 1);
    }
    auto build_tile = [&](int t) {
        if constexpr (TC) {
            const int gt = tc->tbase[g] + t;  // the band's running tile count
            const int slot = gt % kTcSlots;
            // the tile warp has issued the tile's MMAs ...
            bool gave = false;
            for (int it = 0; ld_acquire_cta(&tc->produced[g]) <= gt; ++it) {
                if (it >= A.spin_limit || ((it & 255) == 255 && ld_relaxed(&A.ctl->err) != ERR_NONE)) {
                    set_error(A.ctl, ERR_TIMEOUT, band);
                    gave = true;
                    break;
                }
            }
            // ... and they have completed (the slot's phase of this use)
            for (int it = 0; !gave && !mbar_test(&tc->mbar[g][slot], (uint32_t)(gt / kTcSlots) & 1u); ++it) {
                if (it >= A.spin_limit || ((it & 255) == 255 && ld_relaxed(&A.ctl->err) != ERR_NONE)) {
                    set_error(A.ctl, ERR_TIMEOUT, band);
                    break;
                }
            }
            tc_fence_after();
            float dot[32];
            tc_ld32(tc->tmem + ((uint32_t)(32 * g) << 16) + (uint32_t)((g * kTcSlots + slot) * kTcCols), dot);
            tc_fence_before();
            float* row = tc->tile[g][t % 3][lane];
            const float* yy = tc->yy[g][slot];
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
                const float4 y4 = *reinterpret_cast<const float4*>(yy + j);
                *reinterpret_cast<float4*>(row + j) =
                    make_float4(tc_cost(xxr, y4.x, dot[j]), tc_cost(xxr, y4.y, dot[j + 1]),
                                tc_cost(xxr, y4.z, dot[j + 2]), tc_cost(xxr, y4.w, dot[j + 3]));
            }
            __syncwarp();
            if (lane == 0) st_release_cta(&tc->consumed[g], gt + 1);
        }
    };

    Acc L[R];  // D(p0+k, q-1): the column left of the current one
    int LT[R];
    // KIND_LOCAL: per row of the lane, the lowest value and its first column
    Acc bestv[KIND == KIND_LOCAL ? R : 1];
    int bestq[KIND == KIND_LOCAL ? R : 1];
#pragma unroll
    for (int k = 0; k < (KIND == KIND_LOCAL ? R : 1); ++k) {
        bestv[k] = INF;
        bestq[k] = -1;
    }
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

    // inputs of the next step: the row ring slot of block s (lane 0's row
    // above; every lane reads the same slot) and the frames of block s - lane
    using YF = typename ColFrame<KIND, DIM>::T;
    uint32_t nwd[BW];
    YF ny[U];
    // frames of the lane's block: loaded one step ahead (YPF), or at the step
    // itself for large frames (fewer registers, more resident warps)
    constexpr bool YPF = int_kind(KIND) || DTW_EUC_YPREFETCH != 0 || YW == 0;
    auto load_frames = [&](int cb, YF* dst) {
        if constexpr (YW > 0) {
            const uint32_t* ys = yr + yslot(cb) * YSW;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if constexpr (std::is_same<YF, Frame<KIND, DIM>>::value) dst[u].load_shared(ys + u * YW);
                else dst[u].p = reinterpret_cast<const float*>(ys + u * YW);
            }
        }
    };
    auto fetch = [&](int s) {
        ld_shared_words<BW>(rin + (s & (URS - 1)) * SLOT, nwd);
        const int cb = s - lane;
        if constexpr (TC || !YPF) {
            // tensor-core form: costs come from the tiles; otherwise frames are loaded by the step itself
        } else if constexpr (int_kind(KIND) && U % 4 == 0) {
            uint32_t w[U];
            ld_shared_words<U>(yr + yslot(cb) * YSW, w);
#pragma unroll
            for (int u = 0; u < U; ++u) ny[u].v = (int32_t)w[u];
        } else if constexpr (YW > 0) {
            load_frames(cb, ny);
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = min(max(cb * U + u, 0), Q - 1);
                ny[u].load(sp->colseq, sp->cbase + (long long)sp->cstep * q, A.d);
            }
        }
    };

    bool gave_up = false;
    WaitStats ws;
    Acc end_v = INF;
    int end_t = -1;
    int uroom = URS;  // this warp may write blocks < uroom into rout
    const int nsteps = nblk + 31;

    // the band's last row goes to a ring (the next warp's, or the loader's for the
    // block's last warp) or, without the loader's drain, to global memory
    const bool out_ring = to_ring || (kDr && to_global);
    const bool w31_ring = out_ring && lane == 31, w31_global = !kDr && to_global && lane == 31;
    // warp-uniform: release what the previous groups read and wrote, wait for
    // the blocks this group reads, and for room for the blocks it writes
    int uavail = 0, yavail = 0;  // blocks known to be in the row ring / the frame ring
    auto sync_group = [&](int s0) {
        if (s0 > 0) {
            // One fence of the whole warp, then relaxed counter stores: each is a
            // release of its lane (one fence instead of one per counter).  Row
            // ring: only lane 0's part of each (warp-wide) slot load is used.  Frame
            // ring: every lane reads slots, so the warp synchronises before the
            // fence; every 16 steps (the rings leave room for that staleness).
            // Lane 31 publishes the blocks it wrote.
            const bool yrel = YW > 0 && (s0 & 15) == 0 && s0 > 31;
            if (yrel) __syncwarp();
            asm volatile("fence.acq_rel.cta;" ::: "memory");
            st_relaxed_cta_if(lane == 0 && has_above, &sm.ucons[g], min(s0 + 1, nblk));
            if constexpr (YW > 0) st_relaxed_cta_if(lane == 0 && yrel, &sm.ycons[g], min(s0 - 30, nblk));
            st_relaxed_cta_if(w31_ring && s0 > 31, &sm.uprog[kDr || g + 1 < kG ? g + 1 : g], min(s0 - 31, nblk));
        }
        if (s0 < nblk) {  // lane 0 reads blocks up to s0 + KC (the last one ahead of time)
            const int need = min(s0 + KC + 1, nblk);
            if (has_above && need > uavail)
                uavail = wait_counter(&sm.uprog[g], need, A.ctl, A.spin_limit, band, gave_up, ws);
            if constexpr (YW > 0) {
                if (need > yavail) yavail = wait_counter(&sm.yprog[ys], need, A.ctl, A.spin_limit, band, gave_up, ws);
            }
        }
        if (out_ring) {  // this group writes blocks up to s0 + KC - 32
            const int last = s0 + KC - 32;
            if (last >= uroom)
                uroom = wait_counter(&sm.ucons[g + 1], last + 1 - URS, A.ctl, A.spin_limit, band, gave_up, ws) + URS;
        }
    };

    // checked: some lane may lie outside [0, nblk); capture: some lane may hold the
    // sweep's last block (only groups that reach it take its last cell)
    auto step = [&](int s, auto checked, auto capture) {
        constexpr bool CHECK = decltype(checked)::value;
        constexpr bool CAP = CHECK && decltype(capture)::value;
        uint32_t cw[BW];
#pragma unroll
        for (int i = 0; i < BW; ++i) cw[i] = nwd[i];
        YF yc[U];
        const int cb = s - lane;
        if constexpr (TC) {
        } else if constexpr (YPF) {
#pragma unroll
            for (int u = 0; u < U; ++u) yc[u] = ny[u];
        } else {
            load_frames(cb, yc);
        }
        fetch(s + 1);
        // the row above: lane 0 from the ring, the other lanes by shuffle
        Acc upv[U];
        int upt[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            Acc rv;
            int rt;
            unpack<KIND, NW>(cw + u * NW, rv, rt);
            const Acc sv = shfl_up1(bot[u]);
            upv[u] = lane == 0 ? rv : sv;
            if constexpr (TAG) {
                const int st = __shfl_up_sync(kFull, bott[u], 1);
                upt[u] = lane == 0 ? rt : st;
            } else {
                upt[u] = 0;
            }
        }
        // checked steps: a lane without a block (cb outside [0, nblk)) evaluates its
        // cells on whatever inputs it holds (its rings and frame slots are addressed
        // modulo their sizes) and then resets what it carries to the next step, its
        // left column and its last row, to +infinity: the warp runs the step
        // without a divergent branch.  The tensor-core form indexes its tiles by cb
        // and branches instead.
        const bool act = !CHECK || (unsigned)cb < (unsigned)nblk;
        if (!CHECK || !TC || act) {
            // tensor-core form: the block's two costs from the lane's row of its tile
            float2 tcc = make_float2(0.f, 0.f);
            if constexpr (TC) tcc = *reinterpret_cast<const float2*>(&tc->tile[g][(cb >> 4) % 3][lane][(2 * cb) & 31]);
            Acc rowv[SPECIAL ? R : 1][U];  // the block's cells, for out rows and the last cell
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = cb * U + u;
                Acc a_up = upv[u];
                int t_up = upt[u];
                Acc a_dg = (u == 0) ? dprev : upv[u - 1];
                int t_dg = (u == 0) ? dprevt : upt[u - 1];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    double c = 0.0;
                    if constexpr (TC) c = (double)(u == 0 ? tcc.x : tcc.y);  // cb >= 0 here
                    // edit distance: the diagonal move carries delta, every move the gap
                    const auto cc = [&]() {
                        if constexpr (TC) return c;
                        else if constexpr (edit_kind(KIND)) return egap;
                        else return frame_cost(xr[k], yc[u]);
                    }();
                    const Acc a_dd = [&]() {
                        if constexpr (edit_kind(KIND))
                            return a_dg + edit_delta(xr[k].v, yc[u].v, ematch, esub, egap);
                        else return a_dg;
                    }();
                    const Acc lf = L[k];
                    const Acc m = min3(a_dd, a_up, lf);
                    // integer kind: |x - y| + m in one sum-of-absolute-difference
                    // (m and every accumulated cost are nonnegative and below 2^29)
                    Acc nv;
                    if constexpr (KIND == KIND_ABS) nv = (Acc)__sad(xr[k].v, yc[u].v, (unsigned)m);
                    else nv = m + cc;
                    if constexpr (KIND == KIND_LOCAL) {
                        // local floor (end search), then the row's best node: the first
                        // column attaining the lowest value (q < Q: the last block may
                        // be partial)
                        if (lfloor) nv = min(nv, 0);
                        if ((!CHECK || (act && q < Q)) && nv < bestv[k]) {
                            bestv[k] = nv;
                            bestq[k] = q;
                        }
                    }
                    int t = 0;
                    if constexpr (TAG) {
                        const int t_lf = LT[k];
                        // tag of the backpointer: first minimum among DIAG, UP, LEFT
                        if constexpr (VF) t = (a_dd == m) ? t_dg : ((a_up == m) ? t_up : t_lf);
                        else t = (a_dd == m) ? t_dg : ((lf == m) ? t_lf : t_up);
                        if constexpr (TAGM == 2) t = (p0 + k == tag_row) ? q : t;
                        t_dg = t_lf;
                        t_up = t;
                        LT[k] = t;
                    }
                    if constexpr (SPECIAL) {
                        rowv[k][u] = nv;
                        // the sweep's last cell lies in the lane's last block (a checked
                        // group that reaches it); taken with selects, not a branch
                        if constexpr (CAP) {
                            const bool hit = k == end_k && u == end_u && cb == nblk - 1;
                            end_v = hit ? nv : end_v;
                            end_t = hit ? t : end_t;
                        }
                    }
                    a_dg = lf;
                    a_up = nv;
                    L[k] = nv;
                }
                bot[u] = (!CHECK || TC || act) ? a_up : INF;
                bott[u] = t_up;
            }
            if constexpr (CHECK && !TC) {
#pragma unroll
                for (int k = 0; k < R; ++k) L[k] = act ? L[k] : INF;
            }
            dprev = upv[U - 1];
            dprevt = upt[U - 1];
            if constexpr (SPECIAL) {
                // element offsets stay in 64 bits; only valid rows are stored
                const long long ob = (long long)mo0 * OC + (long long)cb * U * nout;
#pragma unroll
                for (int k = 0; k < R; ++k)
#pragma unroll
                    for (int j = 0; j < U / OC; ++j)
                        store_chunk_if<Acc>(ovalid[k] && act, outp + (ob + (long long)(k + j * nout) * OC),
                                            rowv[k] + j * OC);
            }
        }
        // lane 31: the band's last row over block s-31, for the band below
        // (predicated stores: a checked step outside [0, nblk) stores nothing)
        const int ob = s - 31;
        const bool obok = !CHECK || (ob >= 0 && ob < nblk);
        {
            uint32_t w[BW];
#pragma unroll
            for (int u = 0; u < U; ++u) pack<KIND, NW>(bot[u], bott[u], w + u * NW);
            st_shared_words_if<BW>(w31_ring && obok, rout + (ob & (URS - 1)) * SLOT, w);
            if constexpr (!kDr) {
                unsigned long long* dst = buf + (long long)ob * BW;
#pragma unroll
                for (int i = 0; i < BW / 2; ++i)
                    st_words2_if(w31_global && obok, dst + 2 * i, mkword(w[2 * i], ep_out), mkword(w[2 * i + 1], ep_out));
            }
        }
    };

    // fused split: a band holding split rows counts itself in the sweep's
    // progress word at its end (every lane fences its own stores before the warp
    // barrier, lane 0 then adds, gpu scope)
    sync_group(0);
    fetch(0);
    for (int s0 = 0; s0 < nsteps; s0 += KC) {
        if (s0 > 0) sync_group(s0);
        if (TC && (s0 & 15) == 0 && s0 < nblk) build_tile(s0 >> 4);
        if (s0 >= 31 && s0 + KC < nblk) {
            if constexpr (FULL) {
                // the whole group as straight-line code: steps overlap across it
#pragma unroll
                for (int i = 0; i < KC; ++i) step(s0 + i, std::false_type{}, std::false_type{});
            } else if constexpr (int_kind(KIND)) {
                constexpr int kIU = int_unroll<KIND>();
#pragma unroll kIU
                for (int i = 0; i < KC; ++i) step(s0 + i, std::false_type{}, std::false_type{});
            } else {
                constexpr int kEU = euc_unroll<KIND, DIM>();
#pragma unroll kEU
                for (int i = 0; i < KC; ++i) step(s0 + i, std::false_type{}, std::false_type{});
            }
        } else {
            // the group may run past nsteps: those steps have no lane with a block
            // and store nothing (a per-step test would split the group)
            if (SPECIAL && (s0 + KC < nblk || !need_end)) {
#pragma unroll
                for (int i = 0; i < KC; ++i) step(s0 + i, std::true_type{}, std::false_type{});
            } else {
#pragma unroll
                for (int i = 0; i < KC; ++i) step(s0 + i, std::true_type{}, std::true_type{});
            }
        }
    }
    if (out_ring && lane == 31) st_release_cta(&sm.uprog[g + 1], nblk);
    if constexpr (KIND == KIND_LOCAL) {
        // the band's best node: lowest value, then lowest frame row, then column
        Acc v = INF;
        int bp = INT_MAX, bq = INT_MAX;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            if (p0 + k < rows && bestq[k] >= 0 && bestv[k] < v) {
                v = bestv[k];
                bp = p0 + k;
                bq = bestq[k];
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const Acc ov = __shfl_xor_sync(kFull, v, o);
            const int op = __shfl_xor_sync(kFull, bp, o), oq = __shfl_xor_sync(kFull, bq, o);
            if (ov < v || (ov == v && (op < bp || (op == bp && oq < bq)))) {
                v = ov;
                bp = op;
                bq = oq;
            }
        }
        if (lane == 0 && A.best) {
            int32_t* b = A.best + 4 * (sp->band_begin + band);
            b[0] = v;
            b[1] = bp;
            b[2] = bq;
            b[3] = 1;
        }
    }
    if constexpr (SPECIAL) {
        if (need_end && end_k >= 0 && end_k < R) {
            SweepRes* r = A.res + sweep_idx;
            if constexpr (int_kind(KIND)) r->end_i = end_v;
            else r->end_f = to_double(end_v);
            r->end_tag = end_t;
        }
        if (A.prog != nullptr) {
            int* pw = A.prog + (size_t)sweep_idx * kProgWords;
            const bool holds = out_rows_meet(*sp, band * 32 * R, (band + 1) * 32 * R);
            // the band holding the sweep's last row: its last cell is recorded
            const bool last = (rows - 1) / (32 * R) == band;
            if (holds || last) {
                __threadfence();
                __syncwarp();
                if (lane == 0 && holds) asm volatile("red.relaxed.gpu.global.add.s32 [%0], 1;" ::"l"(pw) : "memory");
                if (lane == 0 && last) asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(pw + 2), "r"(1) : "memory");
            }
        }
    }
    if (lane == 0 && ws.waits) {
        atomicAdd(&A.ctl->resyncs, ws.waits);
        atomicAdd(&A.ctl->polls, ws.polls);
    }
}

// The loader warp.  Round after round it (a) issues, for every frame stream
// with room in its ring, cp.async copies of the next CHB column blocks of the
// sweep's column frames, (b) for warp 0, when its band continues a band of an
// earlier block, polls the next 32 columns of that band's boundary row in
// global memory and copies into row ring 0 the longest run of whole blocks,
// from the first column, whose words all bear the expected epoch, and (c)
// waits for the previous round's copies and publishes them (copies stay one
// round in flight).  Nothing blocks on another
// warp: a round that can do nothing sleeps briefly, and a bounded number of
// idle rounds ends in ERR_TIMEOUT.
template <int KIND, int U, int DIM, int NWMAX, int NW, bool DRAIN>
__device__ __noinline__ void run_loader(const SweepArgs& A, StripSmem<U, NWMAX, FrameWords<KIND, DIM>::v, group_of<KIND>()>& sm) {
    using SM = StripSmem<U, NWMAX, FrameWords<KIND, DIM>::v, group_of<KIND>()>;
    constexpr int YW = FrameWords<KIND, DIM>::v;
    constexpr int SLOT = U * NWMAX;
    constexpr int FB = 4 * YW;  // bytes per frame
    static_assert(32 % U == 0, "a round of 32 boundary columns covers whole blocks");
    constexpr int kG = group_of<KIND>();
    const int lane = threadIdx.x & 31;
    int ynext[kG], yend[kG], ypend[kG];  // blocks issued, to issue, issued in the round in flight
#pragma unroll
    for (int j = 0; j < kG; ++j) {
        const bool head = sm.sweep_of[j] >= 0 && sm.ystream[j] == j;
        ynext[j] = 0;
        ypend[j] = 0;
        yend[j] = (YW > 0 && head) ? A.sweeps[sm.sweep_of[j]].nblk : 0;
    }
    // boundary row for warp 0
    const int si0 = sm.sweep_of[0];
    const Sweep* s0 = si0 >= 0 ? A.sweeps + si0 : nullptr;
    const int uband = s0 ? sm.band_of[0] : 0;
    const int uend = (s0 && uband > 0) ? s0->nblk * U : 0;
    const unsigned long long* ubuf = s0 ? A.bufpool + s0->buf_off : nullptr;
    const uint32_t uep = s0 ? s0->epoch0 + (uint32_t)uband : 0u;  // epoch of the band above
    int unext = 0;
    // the block's last band warp's row, drained into the global boundary row
    // (when its band has a band below): epoch-stamped words, like the band would
    // write them; two payload words per column for float kinds and tag sweeps
    const int sil = sm.sweep_of[kG - 1];
    const Sweep* sl = sil >= 0 ? A.sweeps + sil : nullptr;
    const int dband = sl ? sm.band_of[kG - 1] : 0;
    const bool drain = DRAIN && sl && dband + 1 < sl->nbands && sl->band_begin + dband != A.skip_ticket;
    const int dnblk = drain ? sl->nblk : 0;
    const int dnw = (int_kind(KIND) && (sl == nullptr || sl->tag_row < 0)) ? 1 : 2;
    unsigned long long* dbuf = drain ? A.bufpool + sl->buf_off : nullptr;
    const uint32_t dep = drain ? sl->epoch0 + (uint32_t)dband + 1u : 0u;
    int dnext = 0;  // blocks written to global memory
    bool gave_up = false, inflight = false;
    WaitStats ws;
    unsigned nap = 64;
    for (int idle = 0;;) {
        bool work_left = inflight, progress = false;
        if (dnext < dnblk) {
            work_left = true;
            const int avail = ld_acquire_cta(&sm.uprog[kG]);
            if (avail > dnext) {
                const int b1 = min(avail, dnext + 32 / U);
                const int col = dnext * U + lane;
                if (col < b1 * U) {
                    const uint32_t* src = sm.uring[kG] + ((col / U) & (URS - 1)) * SLOT + (col % U) * dnw;
                    unsigned long long* dst = dbuf + (size_t)col * dnw;
                    for (int i = 0; i < dnw; ++i)
                        asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(dst + i), "l"(mkword(src[i], dep))
                                     : "memory");
                }
                // the warp barrier orders every lane's ring reads before lane 0 frees the slots
                __syncwarp();
                if (lane == 0) st_release_cta(&sm.ucons[kG], b1);
                dnext = b1;
                progress = true;
            }
        }
        int issued[kG];
        if constexpr (YW > 0) {
#pragma unroll
            for (int j = 0; j < kG; ++j) {
                issued[j] = 0;
                if (ynext[j] < yend[j]) {
                    work_left = true;
                    const int b1 = min(ynext[j] + sm.ychb[j], yend[j]);
                    const int YRS = sm.yrs[j];
                    // room: the slowest reader of the stream
                    int rc = 1 << 30;
#pragma unroll
                    for (int g = 0; g < kG; ++g)
                        if (sm.ystream[g] == j && sm.sweep_of[g] >= 0) rc = min(rc, ld_acquire_cta(&sm.ycons[g]));
                    if (b1 <= rc + YRS) {
                        const Sweep* sp = A.sweeps + sm.sweep_of[j];
                        const int Q = sp->Q, cstep = sp->cstep;
                        const long long cbase = sp->cbase;
                        const char* cols = static_cast<const char*>(sp->colseq);
                        uint32_t* yr = sm.yring + (size_t)sm.ybase[j] * SM::YSW;
                        for (int c = ynext[j] * U + lane; c < b1 * U; c += 32) {
                            const char* src = cols + (cbase + (long long)cstep * min(c, Q - 1)) * FB;
                            uint32_t* dst = yr + ((c / U) % YRS) * SM::YSW + (c % U) * YW;
                            if constexpr (FB == 4) {
                                cp_async4(dst, src);
                            } else {
#pragma unroll
                                for (int e = 0; e < FB / 16; ++e) cp_async16(dst + 4 * e, src + 16 * e);
                            }
                        }
                        issued[j] = b1;
                        ynext[j] = b1;
                        progress = true;
                    }
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        if (unext < uend) {
            work_left = true;
            const int nblk = uend / U;
            const int b1 = min((unext + 32) / U, nblk);
            if (b1 <= ld_acquire_cta(&sm.ucons[0]) + URS) {
                const int col = unext + lane;
                unsigned long long w[NW];
                bool ok = col >= uend;
                if (!ok) {
#pragma unroll
                    for (int i = 0; i < NW; ++i) w[i] = ld_word(ubuf + (size_t)col * NW + i);
                    ok = true;
#pragma unroll
                    for (int i = 0; i < NW; ++i) ok = ok && word_epoch(w[i]) == uep;
                }
                // publish the longest run of ready columns from unext, cut to whole
                // blocks: the band below can go on as soon as its next blocks are
                // there, not only when all 32 columns of the window are
                const unsigned bal = __ballot_sync(kFull, ok);
                const int n = (gave_up || bal == kFull) ? 32 : __ffs(~bal) - 1;
                const int newb = min((unext + n) / U, nblk);
                if (newb > unext / U) {
                    const int lim = newb * U;
                    if (col < lim) {
                        uint32_t* dst = sm.uring[0] + ((col / U) & (URS - 1)) * SLOT + (col % U) * NW;
#pragma unroll
                        for (int i = 0; i < NW; ++i) dst[i] = word_payload(w[i]);
                    }
                    // the warp barrier orders every lane's copy before lane 0's release
                    __syncwarp();
                    if (lane == 0) st_release_cta(&sm.uprog[0], newb);
                    unext = lim;
                    progress = true;
                } else {
                    ++ws.polls;
                }
            }
        }
        if constexpr (YW > 0) {
            // the previous round's copies are complete: publish them
            asm volatile("cp.async.wait_group 1;" ::: "memory");
            __syncwarp();  // orders every lane's completed copies before lane 0's releases
            inflight = false;
#pragma unroll
            for (int j = 0; j < kG; ++j) {
                if (ypend[j] > 0 && lane == 0) st_release_cta(&sm.yprog[j], ypend[j]);
                ypend[j] = issued[j];
                inflight = inflight || issued[j] > 0;
            }
        }
        if (!work_left) break;
        if (progress) {
            idle = 0;
            nap = 64;
        } else if (!inflight) {
            if (idle == 0) ++ws.waits;
            if (++idle >= A.spin_limit || ((idle & 63) == 0 && ld_relaxed(&A.ctl->err) != ERR_NONE)) {
                if (!gave_up) set_error(A.ctl, ERR_TIMEOUT, uband);
                gave_up = true;
                // release every ring so that the compute warps finish (on garbage)
                asm volatile("cp.async.wait_group 0;" ::: "memory");
                if (lane == 0) {
#pragma unroll
                    for (int j = 0; j < kG; ++j) st_release_cta(&sm.yprog[j], 1 << 30);
                    st_release_cta(&sm.uprog[0], 1 << 30);
                    st_release_cta(&sm.ucons[kG], 1 << 30);
                }
                break;
            }
            // integer kinds: short steps, the hand-off latency is on the critical
            // path; float kinds: long steps, and the loader shares its scheduler
            // with a band warp, so it backs off (up to 512 ns) while idle
            if constexpr (int_kind(KIND)) {
                __nanosleep(64);
            } else {
                __nanosleep(nap);
                nap = min(2 * nap, 512u);
            }
        }
    }
    if (lane == 0 && ws.waits) {
        atomicAdd(&A.ctl->resyncs, ws.waits);
        atomicAdd(&A.ctl->polls, ws.polls);
    }
}

// The tile warp of the BF16 form (see TcShared).  Once every band warp of the
// ticket has written its rows of operand A, it serves the bands in turn: band
// g's next tile as soon as one of the band's two slots is free -- the column
// frames' FP32 squared norms and BF16 operand B (lane c: column 32t + c), then
// one thread issues the four K = 16 MMAs into the slot's TMEM columns and
// commits them to the slot's mbarrier.  It never waits on one band while
// another could go on; an idle round sleeps briefly and a bounded number of
// them ends in ERR_TIMEOUT.
template <int KIND, int U, int NWMAX>
__device__ __noinline__ void run_tiles(const SweepArgs& A, StripSmem<U, NWMAX, 0, group_of<KIND>()>& sm,
                                       TcShared* tc) {
    constexpr int kG = group_of<KIND>();
    const int lane = threadIdx.x & 31;
    int si = -1;
    unsigned active = 0;
    for (int g = 0; g < kG; ++g) {
        if (sm.sweep_of[g] >= 0) {
            si = sm.sweep_of[g];
            active |= 1u << g;
        }
    }
    if (si < 0) return;
    const Sweep* sp = A.sweeps + si;
    const int Q = sp->Q, ntiles = (Q + kTcCols - 1) / kTcCols;
    const float* colf = static_cast<const float*>(sp->colseq);
    const long long cbase = sp->cbase;
    const int cstep = sp->cstep;
    const int want_a = (int)sm.ticket + 1;
    bool gave_up = false;
    for (int g = 0; g < kG; ++g) {
        if (!((active >> g) & 1u)) continue;
        for (int it = 0; !gave_up && ld_acquire_cta(&tc->a_ready[g]) != want_a; ++it) {
            if (it >= A.spin_limit || ((it & 255) == 255 && ld_relaxed(&A.ctl->err) != ERR_NONE)) {
                set_error(A.ctl, ERR_TIMEOUT, -2);
                gave_up = true;
            }
        }
    }
    const uint32_t a0 = smem_addr(tc->a);
    int next[kTcBands], tb[kTcBands];  // per band: the ticket's next tile, its running-count base
#pragma unroll
    for (int g = 0; g < kTcBands; ++g) {
        tb[g] = tc->tbase[g];
        next[g] = ((active >> g) & 1u) ? 0 : ntiles;
    }
    unsigned nap = 32;
    for (int idle = 0;;) {
        bool left = false, progress = false;
#pragma unroll
        for (int g = 0; g < kTcBands; ++g) {
            if (next[g] >= ntiles) continue;
            left = true;
            const int gt = tb[g] + next[g];
            // the slot's previous tile has been loaded by the band (or the band gave up)
            if (!gave_up && ld_acquire_cta(&tc->consumed[g]) < gt - kTcSlots + 1) continue;
            const int slot = gt % kTcSlots;
            const int q = min(kTcCols * next[g] + lane, Q - 1);
            Frame<KIND_EUC, 64> yf;
            yf.load(colf, cbase + (long long)cstep * q, 64);
            tc->yy[g][slot][lane] = sqnorm<64>(yf.v);
            tc_store_row(tc->b[g][slot], lane, kTcLboB, yf.v);
            fence_proxy_async();  // operand B is read through the async proxy
            __syncwarp();
            if (lane == 0) {
                tc_fence_after();
                const uint32_t b0 = smem_addr(tc->b[g][slot]);
                const uint32_t dt = tc->tmem + (uint32_t)((g * kTcSlots + slot) * kTcCols);
#pragma unroll
                for (int kk = 0; kk < kTcK / 16; ++kk)
                    tc_mma(dt, tc_desc(a0 + (uint32_t)kk * 2 * kTcLboA, kTcLboA, kTcSBO),
                           tc_desc(b0 + (uint32_t)kk * 2 * kTcLboB, kTcLboB, kTcSBO), kk > 0);
                tc_commit(&tc->mbar[g][slot]);
                st_release_cta(&tc->produced[g], gt + 1);
            }
            __syncwarp();
            ++next[g];
            progress = true;
        }
        if (!left) break;
        if (progress) {
            idle = 0;
            nap = 32;
        } else {
            if (++idle >= A.spin_limit || ((idle & 63) == 0 && ld_relaxed(&A.ctl->err) != ERR_NONE)) {
                if (!gave_up) set_error(A.ctl, ERR_TIMEOUT, -2);
                gave_up = true;  // go on without waiting, on garbage
            }
            // a band needs a tile every 16 steps: back off while none is due, so
            // that polling takes few issue slots from the band warp on this SMSP
            __nanosleep(nap);
            nap = min(2 * nap, 1024u);
        }
    }
    // the ticket's MMAs have completed before their slots or operand A are
    // reused (the band warps waited for each; this covers a band that gave up)
#pragma unroll
    for (int g = 0; g < kTcBands; ++g) {
        if (!((active >> g) & 1u) || ntiles == 0) continue;
        const int gl = tb[g] + ntiles - 1;
        for (int it = 0; !mbar_test(&tc->mbar[g][gl % kTcSlots], (uint32_t)(gl / kTcSlots) & 1u); ++it) {
            if (it >= A.spin_limit) {
                set_error(A.ctl, ERR_TIMEOUT, -2);
                break;
            }
        }
    }
}

template <int KIND, int R, int U, int DIM, int NWMAX, int NW, int TAGM, bool VF, bool FULL>
__device__ __forceinline__ void run_band_s(bool special, const Sweep* sp, int si, int band, bool to_ring,
                                           bool to_global, const SweepArgs& A,
                                           StripSmem<U, NWMAX, FrameWords<KIND, DIM>::v, group_of<KIND>()>& sm, int g, TcShared* tc) {
    if (special) run_band<KIND, R, U, DIM, NWMAX, NW, TAGM, VF, true, FULL>(sp, si, band, to_ring, to_global, A, sm, g, tc);
    else run_band<KIND, R, U, DIM, NWMAX, NW, TAGM, VF, false, FULL>(sp, si, band, to_ring, to_global, A, sm, g, tc);
}

// Dynamic shared memory of a block: the strip state, then (tensor-core form)
// the operands, norms, cost tiles and synchronisation of TcShared.
static_assert(kGEucB == kTcBands && kTcBands * 32 == kTcRows, "the BF16 form's block holds the M = 128 rows of one MMA");
template <int KIND, int U, int NWMAX, int DIM>
constexpr size_t strip_smem_bytes(bool tight = false) {
    using SM = StripSmem<U, NWMAX, FrameWords<KIND, DIM>::v, group_of<KIND>()>;
    constexpr size_t base = (sizeof(SM) + 127) & ~(size_t)127;
    // the tight ring: the region's slots beyond kYTight are not allocated
    constexpr size_t cut = ytight_capable(group_of<KIND>(), SM::kBigSlot)
                               ? (size_t)(kYSlotsOf(group_of<KIND>(), SM::kBigSlot) - kYTight) * SM::YSW * 4
                               : 0;
    return base - (tight ? cut : 0) + (KIND == KIND_EUCB ? sizeof(TcShared) + 128 : 0);
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

// The fused split phase: a block that found the ticket queue empty (every band
// of the level is running or done) takes the level's split work items in turn;
// each waits for its columns' split rows (split_item) while the window bands
// finish.
template <int KIND, int DIM, int U, typename SM>
__device__ __noinline__ void split_phase(const SweepArgs& A, SM& sm) {
    const SplitArgs& a = A.split;
    const int n_items = a.n_items >= 0 ? a.n_items : A.ctl->n_items;
    __syncthreads();  // every thread has left the ticket loop (it read sm.ticket)
    for (;;) {
        if (threadIdx.x == 0) {
            sm.ticket = atomicAdd(&A.ctl->split_ticket, 1);
            sm.stop = ld_relaxed(&A.ctl->err) != ERR_NONE;  // outputs of a failed level are not valid
        }
        __syncthreads();
        const int it = (int)sm.ticket;
        const bool stop = sm.stop != 0;
        __syncthreads();
        if (stop || it >= n_items) break;
        split_item<KIND, DIM, true>(a, it, A.prog, A.spin_limit);
    }
}

// TAGS: the launch may contain tagged sweeps (integer kind), whose rows carry
// two payload words per column; untagged integer sweeps use one.  FULL: steady
// groups run fully unrolled (integer variant 3).
template <int KIND, int R, int U, int DIM, bool TAGS, bool FULL>
__device__ __forceinline__ void sweep_body(const SweepArgs& A) {
    constexpr int NWMAX = (!int_kind(KIND) || TAGS) ? 2 : 1;
    constexpr int kG = group_of<KIND>();
    using SM = StripSmem<U, NWMAX, FrameWords<KIND, DIM>::v, group_of<KIND>()>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SM& sm = *reinterpret_cast<SM*>(smem_raw);
    constexpr bool TCK = KIND == KIND_EUCB;
    // the tensor-core state: 128-byte aligned in the shared window (operands)
    TcShared* tcw = nullptr;
    if constexpr (TCK) {
        const unsigned a0 = smem_addr(smem_raw + sizeof(SM));
        tcw = reinterpret_cast<TcShared*>(smem_raw + sizeof(SM) + (((a0 + 127u) & ~127u) - a0));
    }
    int* sweep_of = sm.sweep_of;
    int* band_of = sm.band_of;
    const int warp = threadIdx.x >> 5;
    const int n_sweeps = A.ctl->n_sweeps;
    const long long n_tickets = A.ctl->n_tickets;
    const long long n_bands = A.ctl->n_bands;
    const bool tmap_on = A.ctl->tmap_on != 0 && A.tmap != nullptr;
    // with fewer tickets than blocks only the first n_tickets blocks work: a grid
    // fixed in advance then still puts a level's few strips on separate SMs
    if ((long long)blockIdx.x >= n_tickets) return;
    const bool ytight = ytight_capable(kG, SM::kBigSlot) && A.ytight != 0;
    // tight ring: a second block per SM pays only while tickets are plentiful
    // (three rounds of one block per SM or more); with fewer, the SMs holding
    // two blocks slow their bands and, through the band chain, the whole sweep
    if (ytight && n_tickets < 3LL * A.sms && (int)blockIdx.x >= A.sms) return;
    if constexpr (TCK) {
        // the block's TMEM slots (its tile warp allocates and frees them), the
        // slots' mbarriers (one arrival: the MMAs' commit) and the counters
        if (warp == kG + 1) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tcw->tmem)),
                         "r"(kTcTmemCols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        if (threadIdx.x == 0) {
            for (int g = 0; g < kTcBands; ++g) {
                for (int k = 0; k < kTcSlots; ++k) mbar_init(&tcw->mbar[g][k]);
                tcw->a_ready[g] = 0;
                tcw->produced[g] = 0;
                tcw->consumed[g] = 0;
                tcw->tbase[g] = 0;
                sm.sweep_of[g] = -1;
            }
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            sm.ntiles = 0;
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    for (;;) {
        if (threadIdx.x == 0) {
            sm.ticket = (long long)atomicAdd(&A.ctl->ticket, 1ULL);
            sm.stop = ld_relaxed(&A.ctl->err) != ERR_NONE;
            if constexpr (TCK) {
                // the bands of the previous ticket have consumed all its tiles
                for (int g = 0; g < kTcBands; ++g)
                    if (sm.sweep_of[g] >= 0) tcw->tbase[g] += sm.ntiles;
                sm.ntiles = 0;
            }
        }
        if (threadIdx.x < kG) {
            sm.yprog[threadIdx.x] = 0;
            sm.ycons[threadIdx.x] = 0;
        }
        if (threadIdx.x <= kG) {
            sm.uprog[threadIdx.x] = 0;
            sm.ucons[threadIdx.x] = 0;
        }
        __syncthreads();
        const long long t = sm.ticket;
        if (t >= n_tickets || sm.stop) break;
        if (warp < kG) {
            // the warp's band and sweep, also published for the loader: from the
            // ticket map (group j of one sweep), or consecutive level bands
            int si = -1, band = 0;
            if (tmap_on) {
                const int2 m = A.tmap[t];
                const int b = m.y * kG + warp;
                if (b < A.sweeps[m.x].nbands) {
                    si = m.x;
                    band = b;
                }
            } else {
                const long long gb = t * kG + warp;
                if (gb < n_bands) {
                    si = find_sweep(A.sweeps, n_sweeps, gb);
                    band = (int)(gb - A.sweeps[si].band_begin);
                    // plans with whole groups pad each sweep's bands to a multiple of G
                    if (band >= A.sweeps[si].nbands) si = -1;
                }
            }
            if ((threadIdx.x & 31) == 0) {
                sweep_of[warp] = si;
                band_of[warp] = band;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // frame streams: warps of one sweep share the first one's ring
            int readers[kG] = {};
            for (int g = 0; g < kG; ++g) {
                sm.ystream[g] = (g > 0 && sweep_of[g] >= 0 && sweep_of[g] == sweep_of[g - 1]) ? sm.ystream[g - 1] : g;
                if (sweep_of[g] >= 0) ++readers[sm.ystream[g]];
            }
            int base = 0;
            for (int j = 0; j < kG; ++j) {
                const int w = readers[j] > 0 ? readers[j] : 1;
                sm.ybase[j] = base;
                sm.yrs[j] = yslots(kG, w, SM::kBigSlot, ytight);
                sm.ychb[j] = ychunk(w);
                if (readers[j] > 0) base += yslots(kG, w, SM::kBigSlot, ytight);
            }
            if (base > (ytight ? kYTight : kYSlotsOf(kG, SM::kBigSlot))) {
                // the streams do not fit the frame region (a tight ring, whose
                // tickets must hold one sweep): fail the level, run nothing
                set_error(A.ctl, ERR_CAPACITY, -2);
                for (int g = 0; g < kG; ++g) sweep_of[g] = -1;
            }
            if constexpr (TCK) {
                // tiles of this ticket: the sweep's columns in 32s (every active
                // band warp of a BF16-form ticket belongs to one sweep)
                int si = -1;
                for (int g = 0; g < kG; ++g)
                    if (sweep_of[g] >= 0) si = sweep_of[g];
                sm.ntiles = si >= 0 ? (A.sweeps[si].Q + kTcCols - 1) / kTcCols : 0;
            }
        }
        __syncthreads();
        if (warp < kG) {
            const int si = sweep_of[warp];
            if (si >= 0) {
                const Sweep* sp = A.sweeps + si;
                const int band = band_of[warp];
                const long long gb = sp->band_begin + band;  // level band number
                const int nbands = sp->nbands, rows = sp->rows, tag_row = sp->tag_row;
                const bool below = band + 1 < nbands && gb != A.skip_ticket;
                const bool to_ring = below && warp + 1 < kG;
                const bool to_global = below && warp + 1 == kG;
                const int BR = 32 * R;
                const int b_lo = band * BR, b_hi = b_lo + BR;  // band rows [b_lo, b_hi)
                const bool special = out_rows_meet(*sp, b_lo, b_hi) || (rows - 1 < b_hi);
                if constexpr (!int_kind(KIND)) {
                    run_band_s<KIND, R, U, DIM, NWMAX, 2, 0, true, FULL>(special, sp, si, band, to_ring, to_global, A, sm,
                                                                   warp, tcw);
                } else if (!TAGS || tag_row < 0) {
                    run_band_s<KIND, R, U, DIM, NWMAX, 1, 0, true, FULL>(special, sp, si, band, to_ring, to_global, A, sm,
                                                                   warp, tcw);
                } else if constexpr (TAGS) {
                    const bool vf = sp->axis == 0;
                    if (b_hi <= tag_row) {
                        run_band_s<KIND, R, U, DIM, NWMAX, 2, 0, true, FULL>(special, sp, si, band, to_ring, to_global, A,
                                                                       sm, warp, tcw);
                    } else if (b_lo > tag_row) {
                        if (vf)
                            run_band_s<KIND, R, U, DIM, NWMAX, 2, 1, true, FULL>(special, sp, si, band, to_ring, to_global,
                                                                           A, sm, warp, tcw);
                        else
                            run_band_s<KIND, R, U, DIM, NWMAX, 2, 1, false, FULL>(special, sp, si, band, to_ring, to_global,
                                                                            A, sm, warp, tcw);
                    } else {
                        if (vf)
                            run_band_s<KIND, R, U, DIM, NWMAX, 2, 2, true, FULL>(special, sp, si, band, to_ring, to_global,
                                                                           A, sm, warp, tcw);
                        else
                            run_band_s<KIND, R, U, DIM, NWMAX, 2, 2, false, FULL>(special, sp, si, band, to_ring, to_global,
                                                                            A, sm, warp, tcw);
                    }
                }
            }
        } else if (warp == kG) {
            const int si0 = sweep_of[0];
            if (!int_kind(KIND) || (TAGS && si0 >= 0 && A.sweeps[si0].tag_row >= 0))
                run_loader<KIND, U, DIM, NWMAX, 2, drain_of<KIND, FULL>()>(A, sm);
            else
                run_loader<KIND, U, DIM, NWMAX, 1, drain_of<KIND, FULL>()>(A, sm);
        } else if constexpr (TCK) {
            run_tiles<KIND, U, NWMAX>(A, sm, tcw);
        }
        __syncthreads();
    }
    if constexpr (TCK) {
        // every TMEM load and MMA of the block is complete: free the slots
        tc_fence_before();
        __syncthreads();
        if (warp == kG + 1) {
            tc_fence_after();
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tcw->tmem), "r"(kTcTmemCols)
                         : "memory");
        }
    }
    // (the BF16 form keeps the separate split launch: its split recomputes
    // 64-dimensional BF16 costs, which would raise the whole kernel's registers)
    if constexpr (KIND != KIND_LOCAL && KIND != KIND_EUCB) {
        if (A.prog != nullptr) split_phase<KIND, DIM, U>(A, sm);
    }
}

// The kernel: with the compiler's register count (MB = 0), or with the count
// that lets MB blocks reside on an SM.
template <int KIND, int R, int U, int DIM, bool TAGS, bool FULL>
__global__ void __launch_bounds__(threads_of<KIND>()) sweep_kernel(const __grid_constant__ SweepArgs A) {
    sweep_body<KIND, R, U, DIM, TAGS, FULL>(A);
}
template <int KIND, int R, int U, int DIM, bool TAGS, bool FULL, int MB>
__global__ void __launch_bounds__(threads_of<KIND>(), MB) sweep_kernel_mb(const __grid_constant__ SweepArgs A) {
    sweep_body<KIND, R, U, DIM, TAGS, FULL>(A);
}
template <int KIND, int R, int U, int DIM, bool TAGS, bool FULL, int MB>
constexpr auto sweep_entry() {
    if constexpr (MB > 0)
        return &sweep_kernel_mb<KIND, R, U, DIM, TAGS, FULL, MB>;
    else
        return &sweep_kernel<KIND, R, U, DIM, TAGS, FULL>;
}

// ---------------------------------------------------------------- launchers

// Grid: one block per ticket up to a full persistent grid.  With fewer tickets
// than SMs every block gets an SM of its own, so a level with few bands spreads
// its warps over the schedulers of the whole GPU.
template <int KIND, int R, int U, int DIM, bool TAGS, bool FULL = false, int MB = 0>
static cudaError_t setup_one(int* nb_out, bool tight = false) {
    constexpr int NWMAX = (!int_kind(KIND) || TAGS) ? 2 : 1;
    constexpr size_t smem = strip_smem_bytes<KIND, U, NWMAX, DIM>();
    static_assert(smem <= 227 * 1024, "the block's rings exceed the shared memory of an SM (see yslots)");
    // per device and ring: the attribute is set in (and the occupancy read for)
    // the context of the device that is current; the attribute allows the full
    // region, a launch with the tight ring asks for less
    constexpr int kDevs = 64;
    static std::atomic<int> nb[kDevs][2];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kDevs) return cudaErrorInvalidDevice;
    int v = nb[dev][tight ? 1 : 0].load(std::memory_order_acquire);
    if (v == 0) {
        e = cudaFuncSetAttribute(sweep_entry<KIND, R, U, DIM, TAGS, FULL, MB>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_entry<KIND, R, U, DIM, TAGS, FULL, MB>(), threads_of<KIND>(),
                                                      strip_smem_bytes<KIND, U, NWMAX, DIM>(tight));
        v = n < 1 ? 1 : n;
        nb[dev][tight ? 1 : 0].store(v, std::memory_order_release);
    }
    *nb_out = v;
    return cudaSuccess;
}

template <int KIND, int R, int U, int DIM, bool TAGS, bool FULL = false, int MB = 0>
static cudaError_t launch_one(const SweepArgs& A, int num_sms, long long max_blocks, cudaStream_t st,
                              bool tight = false) {
    constexpr int NWMAX = (!int_kind(KIND) || TAGS) ? 2 : 1;
    const size_t smem = strip_smem_bytes<KIND, U, NWMAX, DIM>(tight);
    int nb = 0;
    cudaError_t e = setup_one<KIND, R, U, DIM, TAGS, FULL, MB>(&nb, tight);
    if (e != cudaSuccess) return e;
    long long grid = (long long)num_sms * nb;
    if (max_blocks > 0 && max_blocks < grid) grid = max_blocks;
    if (max_blocks < 0 || grid < 1) grid = 1;
    SweepArgs B = A;
    B.sms = num_sms;
    B.ytight = tight ? 1 : 0;
    sweep_entry<KIND, R, U, DIM, TAGS, FULL, MB>()<<<(unsigned)grid, threads_of<KIND>(), smem, st>>>(B);
    return cudaGetLastError();
}

// Variants: integer |x-y| with an R x U block per lane and step (tagged rows
// allowed or not), Euclidean d=12 (R=2, U=2) and any other d read from memory
// (R=2, U=2).  A lane's R x U block is a small wavefront of its own: its
// anti-diagonals give the scheduler independent cells, and the per-step
// hand-off work (shuffles, ring, boundary stores) is paid once per block.
constexpr int kIntR = DTW_INT_R, kIntU = DTW_INT_U;
constexpr int kEucR = DTW_EUC_R, kEucU = DTW_EUC_U;
// Integer variants (selected at run time, e.g. by the autotuner): rows per lane
// (variant 3: the default lane block with fully unrolled steady groups).
constexpr int kIntRVar[kSweepVariants] = {kIntR, 2, 8, kIntR};
int sweep_block_cols(int kind, int d, int variant) { return int_kind(kind) ? kIntU : (d == 12 ? kEucU : 2); }
int sweep_band_rows(int kind, int d, int variant) {
    if (kind == KIND_ABS) return 32 * kIntRVar[(unsigned)variant < (unsigned)kSweepVariants ? variant : 0];
    if (edit_kind(kind)) return 32 * kIntR;
    return d == 12 ? 32 * kEucR : (d == 64 ? 32 : 64);
}
bool sweep_whole_groups(int kind, int d) {
    return kind == KIND_EUCB || ((kind == KIND_EUC || kind == KIND_EUCF) && d == 64);
}
int sweep_group_bands(int kind) {
    return int_kind(kind) ? group_of<KIND_ABS>() : (kind == KIND_EUCB ? group_of<KIND_EUCB>() : group_of<KIND_EUC>());
}

cudaError_t sweep_prepare(int kind, int d, bool tags, int variant) {
    int nb = 0;
    if (kind == KIND_ABS) {
        if (variant == 1) return tags ? setup_one<KIND_ABS, 2, kIntU, 1, true>(&nb) : setup_one<KIND_ABS, 2, kIntU, 1, false>(&nb);
        if (variant == 2) return tags ? setup_one<KIND_ABS, 8, kIntU, 1, true>(&nb) : setup_one<KIND_ABS, 8, kIntU, 1, false>(&nb);
        if (variant == 3)
            return tags ? setup_one<KIND_ABS, kIntR, kIntU, 1, true, true>(&nb)
                        : setup_one<KIND_ABS, kIntR, kIntU, 1, false, true>(&nb);
        if (tags) return setup_one<KIND_ABS, kIntR, kIntU, 1, true>(&nb);
        return setup_one<KIND_ABS, kIntR, kIntU, 1, false>(&nb);
    }
    if (kind == KIND_EDIT) return tags ? setup_one<KIND_EDIT, kIntR, kIntU, 1, true>(&nb)
                                       : setup_one<KIND_EDIT, kIntR, kIntU, 1, false>(&nb);
    if (kind == KIND_LOCAL) return setup_one<KIND_LOCAL, kIntR, kIntU, 1, false>(&nb);
    if (kind == KIND_EUCB) return setup_one<KIND_EUCB, 1, 2, 64, false>(&nb);
    if (kind == KIND_EUCF) {
        if (d == 12 && variant == 1) return setup_one<KIND_EUCF, kEucR, kEucU, 12, false, false, kEucMinB>(&nb);
        if (d == 12) return setup_one<KIND_EUCF, kEucR, kEucU, 12, false>(&nb);
        if (d == 64) return setup_one<KIND_EUCF, 1, 2, 64, false>(&nb, variant == 1);
        return setup_one<KIND_EUCF, 2, 2, 0, false>(&nb);
    }
    if (d == 12 && variant == 1) return setup_one<KIND_EUC, kEucR, kEucU, 12, false, false, kEucMinB>(&nb);
    if (d == 12) return setup_one<KIND_EUC, kEucR, kEucU, 12, false>(&nb);
    if (d == 64) return setup_one<KIND_EUC, 1, 2, 64, false>(&nb, variant == 1);
    return setup_one<KIND_EUC, 2, 2, 0, false>(&nb);
}

int sweep_variant_for(int kind, int d, int variant, long long tickets0, int num_sms) {
    if (int_kind(kind)) return variant;
    if (kind != KIND_EUC && kind != KIND_EUCF) return 0;
    // d = 64: the tight frame ring (two blocks per SM) when the first level has
    // three rounds of tickets for one block per SM or more
    if (d == 64) return tickets0 >= 3LL * num_sms ? 1 : 0;
    if (d != 12) return 0;
    int nb = 0;
    const cudaError_t e = kind == KIND_EUC ? setup_one<KIND_EUC, kEucR, kEucU, 12, false>(&nb)
                                           : setup_one<KIND_EUCF, kEucR, kEucU, 12, false>(&nb);
    if (e != cudaSuccess) return 0;  // the launch reports the error
    return tickets0 > (long long)nb * num_sms ? 1 : 0;
}

cudaError_t launch_sweep(int kind, int d, bool tags, const SweepArgs& A, int num_sms, long long max_blocks,
                         cudaStream_t st, int variant) {
    if (kind == KIND_ABS) {
        if (variant == 1)
            return tags ? launch_one<KIND_ABS, 2, kIntU, 1, true>(A, num_sms, max_blocks, st)
                        : launch_one<KIND_ABS, 2, kIntU, 1, false>(A, num_sms, max_blocks, st);
        if (variant == 2)
            return tags ? launch_one<KIND_ABS, 8, kIntU, 1, true>(A, num_sms, max_blocks, st)
                        : launch_one<KIND_ABS, 8, kIntU, 1, false>(A, num_sms, max_blocks, st);
        if (variant == 3)
            return tags ? launch_one<KIND_ABS, kIntR, kIntU, 1, true, true>(A, num_sms, max_blocks, st)
                        : launch_one<KIND_ABS, kIntR, kIntU, 1, false, true>(A, num_sms, max_blocks, st);
        if (tags) return launch_one<KIND_ABS, kIntR, kIntU, 1, true>(A, num_sms, max_blocks, st);
        return launch_one<KIND_ABS, kIntR, kIntU, 1, false>(A, num_sms, max_blocks, st);
    }
    if (kind == KIND_EDIT)
        return tags ? launch_one<KIND_EDIT, kIntR, kIntU, 1, true>(A, num_sms, max_blocks, st)
                    : launch_one<KIND_EDIT, kIntR, kIntU, 1, false>(A, num_sms, max_blocks, st);
    if (kind == KIND_LOCAL) return launch_one<KIND_LOCAL, kIntR, kIntU, 1, false>(A, num_sms, max_blocks, st);
    if (kind == KIND_EUCB) return launch_one<KIND_EUCB, 1, 2, 64, false>(A, num_sms, max_blocks, st);
    if (kind == KIND_EUCF) {
        if (d == 12 && variant == 1)
            return launch_one<KIND_EUCF, kEucR, kEucU, 12, false, false, kEucMinB>(A, num_sms, max_blocks, st);
        if (d == 12) return launch_one<KIND_EUCF, kEucR, kEucU, 12, false>(A, num_sms, max_blocks, st);
        if (d == 64) return launch_one<KIND_EUCF, 1, 2, 64, false>(A, num_sms, max_blocks, st, variant == 1);
        return launch_one<KIND_EUCF, 2, 2, 0, false>(A, num_sms, max_blocks, st);
    }
    if (d == 12 && variant == 1)
        return launch_one<KIND_EUC, kEucR, kEucU, 12, false, false, kEucMinB>(A, num_sms, max_blocks, st);
    if (d == 12) return launch_one<KIND_EUC, kEucR, kEucU, 12, false>(A, num_sms, max_blocks, st);
    // d = 64: one row per lane (its frame in registers), column frames read in place
    if (d == 64) return launch_one<KIND_EUC, 1, 2, 64, false>(A, num_sms, max_blocks, st, variant == 1);
    return launch_one<KIND_EUC, 2, 2, 0, false>(A, num_sms, max_blocks, st);
}

}  // namespace dtwb
