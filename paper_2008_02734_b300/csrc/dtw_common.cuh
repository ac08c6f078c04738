// Device-side types and helpers shared by the kernels of the library.
//
// Frames (Section 2.1): pair b aligns X (M frames) with Y (N frames).  A "box" is
// the sub-problem [i0, i0+H) x [j0, j0+W) of one pair whose first and last cells
// are known to lie on the optimal path (Algorithm 2's recursion).  A box is swept
// in a "frame" (p, q): p runs along the split axis (X rows when H >= W, else Y
// rows), q along the other axis, and a backward sweep reverses both (the
// reversed series X_R, Y_R of Algorithm 2, done by index arithmetic).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace dtwb {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

// Cost kinds (low byte of the ABI's cost_kind).
constexpr int KIND_EUC = 0;  // Euclidean distance of FP32 frames, FP64 accumulation
constexpr int KIND_ABS = 1;  // |x - y| of int32 samples, exact int32 accumulation
constexpr int KIND_EUCF = 2; // Euclidean distance of FP32 frames, compensated FP32-pair accumulation
constexpr int KIND_EUCB = 3; // Euclidean distance in the expanded form with BF16 products (tensor-core
                             // cost tiles), compensated FP32-pair accumulation; d = 64
// Weighted edit distance of int32 symbol sequences (Section 5 names it as a
// problem of the same DP design), run as the same recursion on its node grid:
// the pair handed to the kernels is the two sequences with a sentinel symbol at
// both ends (frames 0 .. M+1), M+1 x N+1 "cells" (the nodes), and a cell update
//   E = min(E_diag + delta, E_up, E_left) + gap,  delta = s(x, y) - gap,
// with s(x, y) = 0 for equal symbols, else sub.  The first node of a box takes
// E = s of its own symbols (the corner is 0), a constant that every value of
// the box carries; the backward sweep reads its symbols one index further (the
// step into reversed node p consumes forward symbol p + 1).  The split sums
// F + B with no cell term.
constexpr int KIND_EDIT = 4;
// Local alignment (Smith-Waterman, named in Section 5 beside edit distance):
// the edit update on the node grid with scores turned into costs (match cost
// -match, mismatch cost mismatch, gap cost gap), and for the end search the
// local floor E = min(E, 0) (H = max(H, 0)).  Its sweeps also keep each band's
// best node (lowest value, then first in row-major order of the sweep frame).
constexpr int KIND_LOCAL = 5;
__host__ __device__ constexpr bool int_kind(int k) { return k == KIND_ABS || k == KIND_EDIT || k == KIND_LOCAL; }
__host__ __device__ constexpr bool edit_kind(int k) { return k == KIND_EDIT || k == KIND_LOCAL; }
// The sentinel symbol at both ends of an edit pair (inputs may not contain it).
constexpr int32_t kEditPad = (int32_t)0x80000000;

// "Infinity" of the int32 accumulator: above any reachable cost (the host
// guarantees max C * (M+N-1) < 2^29) and far from overflow when C is added.
constexpr int32_t kIntInf = 0x3FFFFFFF;

// Device error codes (stored in LevelCtl::err; first error wins).
constexpr int ERR_NONE = 0;
constexpr int ERR_TIMEOUT = 1;     // a bounded wait gave up
constexpr int ERR_CONSIST = 2;     // a box's swept cost differs from its known cost
constexpr int ERR_PATH = 3;        // the assembled path is not a warping path
constexpr int ERR_OVERFLOW = 4;    // integer accumulator range exceeded
constexpr int ERR_CAPACITY = 5;    // a level needs more workspace than reserved

struct PairDesc {
    const void* X;      // M*d frames
    const void* Y;      // N*d frames
    int32_t M, N;
    int32_t row_off;    // offset of the pair's rows in the per-row path arrays
    int32_t flags;
    int32_t* path;      // device path buffer, 2*(M+N-1) int32
    int32_t esub, egap; // KIND_EDIT / KIND_LOCAL: substitution and gap costs
    int32_t ematch;     // and the cost of a match (0 for edit distance, negative for local scores)
};

struct PairRes {
    long long cost_i;   // exact D* (KIND_ABS)
    double cost_f;      // D* (KIND_EUC)
    int32_t K;          // path length
    int32_t pad;
};

constexpr int BOX_ROOT = 1;  // the pair's whole problem: its result is the pair's D*
constexpr int BOX_TAG = 2;   // integer box whose split rows all tied: use a tagged sweep

struct Box {
    int32_t pair, i0, j0, H, W, flags;
    long long known_i;  // optimal cost of the box if known (KIND_ABS), else -1
    double known_f;     // optimal cost of the box (KIND_EUC), NaN if unknown
};

// Columns of a split row handled by one split work item (one 256-thread block).
#ifndef DTW_SPLIT_CHUNK
#define DTW_SPLIT_CHUNK 256
#endif
constexpr int kSplitChunk = DTW_SPLIT_CHUNK;
// Columns of one split work item of a box with nw windows of split rows: the
// item covers one window, nw chunks wide, so that a box has about as many items
// as with a single window.
__host__ __device__ __forceinline__ int split_item_cols(int nw) { return kSplitChunk * (nw > 1 ? nw : 1); }

// Half-width of a window of split rows written by forward/backward sweeps of
// integer boxes: rows r-kSplitHalo .. r+kSplitHalo around a split row r.
constexpr int kSplitHalo = 4;
constexpr int kSplitRowsMax = 2 * kSplitHalo + 1;

// Several split rows per box (Lemma 1 holds for each of them): a box's two sweeps
// may end on up to kSplitWinMax equally spaced windows of split rows, at most
// kOutRowsMax rows in all, each window kWinGap rows or more from the next (more
// than the rows a lane of any sweep variant owns, so that a lane's rows meet one
// window at most).
constexpr int kSplitWinMax = 15;
constexpr int kOutRowsMax = 64;
constexpr int kWinGap = 8;

// One wavefront sweep over frame rows [0, rows) x frame columns [0, Q).  16-byte
// aligned (144 bytes): the plan writes a level's descriptors with 16-byte stores.
struct alignas(16) Sweep {
    const void* rowseq;  // features indexed by frame row p: rowseq[rbase + rstep*p]
    const void* colseq;  // features indexed by frame column q: colseq[cbase + cstep*q]
    int32_t rbase, rstep, cbase, cstep;
    int32_t box;         // index in the level's box array
    int32_t dir;         // 0 forward from the box's first cell, 1 backward from its last
    int32_t axis;        // 0: p runs along X; 1: p runs along Y
    int32_t rows;        // frame rows swept (0: empty slot)
    int32_t Q;           // frame columns
    int32_t nblk;        // column blocks of the sweep's kernel variant
    int32_t out_row0;    // first frame row copied to the out pool (first row of the first window)
    int32_t nout;        // rows copied (0: none): onw windows of owin rows
    int32_t onw;         // windows of split rows
    int32_t owin;        // rows per window
    int32_t ospace;      // frame rows from one window's first row to the next one's
    int32_t tag_row;     // frame row where split tags start (-1: untagged sweep)
    int32_t nbands;
    uint32_t epoch0;     // band b stamps its boundary words with epoch0 + b + 1
    int32_t ostride;     // out-row stride (columns padded to whole blocks)
    int32_t item0;       // first split work item of the box (forward slot only)
    int32_t nitems;      // split work items of the box: column chunks of its split rows (forward slot only)
    long long band_begin;  // level band number of the sweep's first band
    long long buf_off;     // boundary-row pool offset, in 64-bit words (1 or 2 per column)
    long long out_off;     // out pool offset: nout rows of ostride values, in the sweep's own frame order
    int32_t esub, egap;    // KIND_EDIT / KIND_LOCAL: substitution and gap costs
    int32_t ematch;        // match cost
    int32_t floor;         // KIND_LOCAL: the local floor E = min(E, 0) applies
};

struct SweepRes {
    long long end_i;  // accumulated cost at the sweep's last cell (KIND_ABS)
    double end_f;     // (KIND_EUC)
    int32_t end_tag;  // split tag carried to the last cell (tag sweeps)
    int32_t pad;
};

// Control block of a call, in device memory.
struct LevelCtl {
    unsigned long long ticket;   // next ticket (a group of consecutive bands) of the current sweep launch
    long long n_tickets;         // tickets in the current level
    long long n_bands;           // bands in the current level
    int32_t n_cur;               // boxes of the current level (set by the plan)
    int32_t n_items;             // split work items of the current level
    int32_t n_sweeps;
    int32_t n_next;              // boxes appended to the next level
    int32_t n_base;              // boxes appended to the base list (all levels)
    int32_t err;                 // first device error (ERR_*)
    int32_t err_info;
    uint32_t epoch_base;         // next unused boundary-word epoch (never reused)
    unsigned long long sweep_cells;
    unsigned long long tag_cells;
    unsigned long long base_cells;
    long long need_buf;          // pool words the current level needs
    long long retag;             // boxes sent back for a tagged sweep
    unsigned long long resyncs;  // prefetch-ring refills in the sweeps
    unsigned long long polls;    // failed polls of boundary words
    int32_t levels;              // levels planned on the device (graph-driven level loop)
    int32_t tmap_on;             // the current level's tickets follow the ticket map (group-major order)
    int32_t split_ticket;        // next split work item of the sweep kernel's split phase
    int32_t n_tag;               // boxes of the current level that take a tagged sweep (set by the plan)
};

// ---------------------------------------------------------------- memory order

__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Boundary words: a 64-bit word carries a 32-bit payload (low half) and the
// epoch of the band that wrote it (high half).  A single aligned 64-bit relaxed
// access is single-copy atomic, so a reader that sees the expected epoch holds
// that band's payload -- no fence or flag is needed, and stale words from earlier
// bands, levels or calls (smaller epochs) are simply not accepted.
__device__ __forceinline__ void st_word(unsigned long long* p, uint32_t payload, uint32_t epoch) {
    const unsigned long long w = ((unsigned long long)epoch << 32) | payload;
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__device__ __forceinline__ unsigned long long ld_word(const unsigned long long* p) {
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
    return w;
}

__device__ __forceinline__ uint32_t word_epoch(unsigned long long w) { return (uint32_t)(w >> 32); }
__device__ __forceinline__ uint32_t word_payload(unsigned long long w) { return (uint32_t)w; }

__device__ __forceinline__ void set_error(LevelCtl* ctl, int code, int info) {
    if (atomicCAS(&ctl->err, ERR_NONE, code) == ERR_NONE) ctl->err_info = info;
}

// ---------------------------------------------------------------- accumulators

// Compensated FP32 accumulator (the DTW_DP_F32_KAHAN form): an unevaluated sum
// hi + lo of two FP32 values with |lo| <= ulp(hi)/2, so about 48 significant
// bits.  A frame cost c (an FP32 value) is added with TwoSum (the exact rounding
// error of hi + c) followed by a renormalisation; the minimum compares (hi, lo)
// lexicographically, which orders normalised pairs exactly.  "Infinity" is a
// large finite hi, so that no operation ever meets inf - inf.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_add(DF a, float c) {
    const float s = __fadd_rn(a.hi, c);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(c, bb));
    const float t = __fadd_rn(e, a.lo);
    const float hi = __fadd_rn(s, t);
    return DF{hi, __fsub_rn(t, __fsub_rn(hi, s))};
}
__device__ __forceinline__ DF operator+(DF a, double c) { return df_add(a, (float)c); }  // c: a widened FP32 cost
__device__ __forceinline__ bool operator==(DF a, DF b) { return a.hi == b.hi && a.lo == b.lo; }
// lexicographic order of normalised pairs; bitwise logic: no short-circuit branches
__device__ __forceinline__ bool operator<(DF a, DF b) { return (a.hi < b.hi) | ((a.hi == b.hi) & (a.lo < b.lo)); }
__device__ __forceinline__ DF df_min(DF a, DF b) {
    const bool lt = b < a;
    return DF{lt ? b.hi : a.hi, lt ? b.lo : a.lo};
}
__device__ __forceinline__ DF min3(DF a, DF b, DF c) { return df_min(df_min(a, b), c); }
__device__ __forceinline__ DF acc_min(DF a, DF b) { return df_min(a, b); }
__device__ __forceinline__ double acc_min(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ int32_t acc_min(int32_t a, int32_t b) { return a < b ? a : b; }
__device__ __forceinline__ double to_double(DF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double to_double(double a) { return a; }
__device__ __forceinline__ double to_double(int32_t a) { return (double)a; }

// Warp shuffle of an accumulator from the lane below (lane - 1).
__device__ __forceinline__ int32_t shfl_up1(int32_t v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_up1(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ DF shfl_up1(DF v) {
    return DF{__shfl_up_sync(0xffffffffu, v.hi, 1), __shfl_up_sync(0xffffffffu, v.lo, 1)};
}
__device__ __forceinline__ int32_t shfl_down(int32_t v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ DF shfl_down(DF v, int o) {
    return DF{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}

template <int KIND> struct AccOf;
template <> struct AccOf<KIND_ABS> {
    using T = int32_t;
    static __device__ __forceinline__ T inf() { return kIntInf; }
    static __device__ __forceinline__ T zero() { return 0; }
};
template <> struct AccOf<KIND_EUC> {
    using T = double;
    static __device__ __forceinline__ T inf() { return __longlong_as_double(0x7ff0000000000000LL); }
    static __device__ __forceinline__ T zero() { return 0.0; }
};
template <> struct AccOf<KIND_EUCF> {
    using T = DF;
    static __device__ __forceinline__ T inf() { return DF{1e30f, 0.f}; }
    static __device__ __forceinline__ T zero() { return DF{0.f, 0.f}; }
};
template <> struct AccOf<KIND_EUCB> : AccOf<KIND_EUCF> {};
template <> struct AccOf<KIND_EDIT> : AccOf<KIND_ABS> {};
template <> struct AccOf<KIND_LOCAL> : AccOf<KIND_ABS> {};

__device__ __forceinline__ int32_t min3(int32_t a, int32_t b, int32_t c) { return __vimin3_s32(a, b, c); }
// Accumulated costs are sums of nonnegative frame costs (or +infinity), and for
// nonnegative doubles the IEEE-754 bit pattern, read as a signed 64-bit integer,
// orders exactly like the value.  The minimum is therefore taken with integer
// compares and selects, which run on the full-rate integer pipe, instead of
// FP64 minimum instructions, which share the narrow FP64 pipe with the additions.
__device__ __forceinline__ double min3(double a, double b, double c) {
    const long long x = __double_as_longlong(a), y = __double_as_longlong(b), z = __double_as_longlong(c);
    const long long m = x < y ? x : y;
    return __longlong_as_double(m < z ? m : z);
}

// ---------------------------------------------------------------- frame features

// A frame held in registers.  DIM > 0: compile-time dimension; the int kind has DIM 1.
template <int KIND, int DIM> struct Frame;

template <> struct Frame<KIND_ABS, 1> {
    int32_t v;
    __device__ __forceinline__ void load(const void* base, long long idx, int /*d*/) {
        v = __ldg(static_cast<const int32_t*>(base) + idx);
    }
    __device__ __forceinline__ void load_shared(const void* p) { v = *static_cast<const int32_t*>(p); }
};
template <> struct Frame<KIND_EDIT, 1> : Frame<KIND_ABS, 1> {};
template <> struct Frame<KIND_LOCAL, 1> : Frame<KIND_ABS, 1> {};

template <int DIM> struct Frame<KIND_EUC, DIM> {
    float v[DIM];
    __device__ __forceinline__ void load(const void* base, long long idx, int /*d*/) {
        const float* p = static_cast<const float*>(base) + idx * DIM;
        if constexpr (DIM % 4 == 0) {
            const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
            for (int e = 0; e < DIM / 4; ++e) {
                float4 t = __ldg(p4 + e);
                v[4 * e] = t.x;
                v[4 * e + 1] = t.y;
                v[4 * e + 2] = t.z;
                v[4 * e + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int e = 0; e < DIM; ++e) v[e] = __ldg(p + e);
        }
    }
    __device__ __forceinline__ void load_shared(const void* ps) {
        const float* p = static_cast<const float*>(ps);
        if constexpr (DIM % 4 == 0) {
#pragma unroll
            for (int e = 0; e < DIM / 4; ++e) {
                const float4 t = reinterpret_cast<const float4*>(p)[e];
                v[4 * e] = t.x;
                v[4 * e + 1] = t.y;
                v[4 * e + 2] = t.z;
                v[4 * e + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int e = 0; e < DIM; ++e) v[e] = p[e];
        }
    }
};

// Runtime dimension: the frame stays in global memory (read through L1).
template <> struct Frame<KIND_EUC, 0> {
    const float* p;
    int d;
    __device__ __forceinline__ void load(const void* base, long long idx, int dd) {
        d = dd;
        p = static_cast<const float*>(base) + idx * dd;
    }
    __device__ __forceinline__ void load_shared(const void*) {}
};

// The compensated kind reads the same frames (its costs are the same FP32 values).
template <int DIM> struct Frame<KIND_EUCF, DIM> : Frame<KIND_EUC, DIM> {};
// The BF16 form reads the same FP32 frames; its cost is the expanded form below.
template <int DIM> struct Frame<KIND_EUCB, DIM> : Frame<KIND_EUC, DIM> {};

// Expanded-form cost of the BF16 form: sqrt(max(0, |x|^2 + |y|^2 - 2 x.y)) with
// the squared norms summed in FP32 from the FP32 coordinates (in coordinate
// order) and the dot product of the BF16-rounded coordinates accumulated in FP32
// -- the products of two BF16 values are exact in FP32, as in the tensor-core
// tiles of the sweep, which accumulate the same products in their own order.
__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float expanded_cost(float xx, float yy, float dot) {
    const float t = __fmaf_rn(-2.f, dot, __fadd_rn(xx, yy));
    return __fsqrt_rn(fmaxf(t, 0.f));
}
template <int DIM>
__device__ __forceinline__ float sqnorm(const float* v) {
    float s = 0.f;
#pragma unroll
    for (int e = 0; e < DIM; ++e) s = __fmaf_rn(v[e], v[e], s);
    return s;
}

// Frame cost C (Section 2.1): |x-y|, or the Euclidean distance (Section 4.1)
// evaluated in FP32 (sum of squares with FMA, square root by cost_sqrt) and widened.
__device__ __forceinline__ int32_t frame_cost(const Frame<KIND_ABS, 1>& a, const Frame<KIND_ABS, 1>& b) {
    return abs(a.v - b.v);
}
// Edit distance: no cost sits on a node, so the split sums F + B alone; the
// sweeps and the base case use edit_delta and the gap instead.
__device__ __forceinline__ int32_t frame_cost(const Frame<KIND_EDIT, 1>&, const Frame<KIND_EDIT, 1>&) { return 0; }
__device__ __forceinline__ int32_t frame_cost(const Frame<KIND_LOCAL, 1>&, const Frame<KIND_LOCAL, 1>&) { return 0; }
__device__ __forceinline__ int32_t edit_delta(int32_t x, int32_t y, int32_t match, int32_t sub, int32_t gap) {
    return (x == y ? match : sub) - gap;
}

// Square root of a frame cost's sum of squares: the hardware approximation
// (sqrt.approx.f32, one instruction, within 2 ulp; exact at +0 and +infinity),
// or with DTW_EUC_SQRT_APPROX=0 the correctly rounded square root, several
// instructions with a slow-path branch.  The approximation adds at most about
// 2.4e-7 relative to a cost, the size of the FP32 sum of squares' own rounding,
// far inside the 1e-6 tolerance; every kernel evaluates costs through here, so
// the sweeps, the split and the base case see the same cost of a cell.
#ifndef DTW_EUC_SQRT_APPROX
#define DTW_EUC_SQRT_APPROX 1
#endif
__device__ __forceinline__ float cost_sqrt(float s) {
#if DTW_EUC_SQRT_APPROX
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(s));
    return r;
#else
    return __fsqrt_rn(s);
#endif
}

// Exact FP32 -> FP64 widening of a frame cost with integer operations (the
// conversion instruction would occupy the narrow FP64 pipe).  A Euclidean frame
// cost is +0, a positive normal FP32 value (the square root of even the smallest
// subnormal sum is normal) or +infinity: shifting the bit pattern into the
// double's fields and rebasing the exponent (bias 127 -> 1023) is exact.
__device__ __forceinline__ double widen_cost(float c) {
    const unsigned u = __float_as_uint(c);
    const unsigned long long b = ((unsigned long long)u << 29) + (896ULL << 52);
    const long long r = u == 0u ? 0LL : (u >= 0x7f800000u ? 0x7ff0000000000000LL : (long long)b);
    return __longlong_as_double(r);
}

// Fixed even dimension: packed FP32x2 arithmetic (one instruction per two
// dimensions for the difference and one for the square-accumulate), two partial
// sums over the even and the odd coordinates, added at the end.
// Dimensions that are multiples of 8: four packed partial sums (coordinates
// e, e+1 go to sum (e/2) mod 4), so the accumulation chain is a quarter as long;
// the sums are combined as ((s0 + s1) + (s2 + s3)) and then x + y.  Every kernel
// evaluates a cost in exactly this order.
template <int DIM>
__device__ __forceinline__ float sumsq8(const float* a, const float* b) {
    float2 s[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) s[i] = make_float2(0.f, 0.f);
    const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
    for (int e = 0; e < DIM; e += 2) {
        const float2 t = __ffma2_rn(make_float2(b[e], b[e + 1]), m1, make_float2(a[e], a[e + 1]));
        s[(e / 2) & 3] = __ffma2_rn(t, t, s[(e / 2) & 3]);
    }
    const float2 r = __fadd2_rn(__fadd2_rn(s[0], s[1]), __fadd2_rn(s[2], s[3]));
    return r.x + r.y;
}

template <int DIM>
__device__ __forceinline__ double frame_cost(const Frame<KIND_EUC, DIM>& a, const Frame<KIND_EUC, DIM>& b) {
    if constexpr (DIM % 8 == 0) {
        return widen_cost(cost_sqrt(sumsq8<DIM>(a.v, b.v)));
    } else if constexpr (DIM % 2 == 0) {
        float2 s = make_float2(0.f, 0.f);
        const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
        for (int e = 0; e < DIM; e += 2) {
            const float2 t = __ffma2_rn(make_float2(b.v[e], b.v[e + 1]), m1, make_float2(a.v[e], a.v[e + 1]));
            s = __ffma2_rn(t, t, s);
        }
        return widen_cost(cost_sqrt(s.x + s.y));
    } else {
        float s = 0.f;
#pragma unroll
        for (int e = 0; e < DIM; ++e) {
            float t = a.v[e] - b.v[e];
            s = fmaf(t, t, s);
        }
        return widen_cost(cost_sqrt(s));
    }
}

__device__ __forceinline__ double frame_cost(const Frame<KIND_EUC, 0>& a, const Frame<KIND_EUC, 0>& b) {
    float s = 0.f;
    for (int e = 0; e < a.d; ++e) {
        float t = __ldg(a.p + e) - __ldg(b.p + e);
        s = fmaf(t, t, s);
    }
    return widen_cost(cost_sqrt(s));
}

template <int DIM>
__device__ __forceinline__ double frame_cost(const Frame<KIND_EUCB, DIM>& a, const Frame<KIND_EUCB, DIM>& b) {
    float dot = 0.f;
#pragma unroll
    for (int e = 0; e < DIM; ++e) dot = __fmaf_rn(bf16_round(a.v[e]), bf16_round(b.v[e]), dot);
    return widen_cost(expanded_cost(sqnorm<DIM>(a.v), sqnorm<DIM>(b.v), dot));
}

// A column frame read in place (shared memory), for large fixed dimensions whose
// frames do not fit in registers next to the row frames.
template <int DIM>
struct FrameRef {
    const float* p;
};

template <int DIM>
__device__ __forceinline__ double frame_cost(const Frame<KIND_EUC, DIM>& a, const FrameRef<DIM>& b) {
    static_assert(DIM % 8 == 0, "in-place frames use the eight-coordinate order");
    float y[DIM];
#pragma unroll
    for (int e = 0; e < DIM; e += 4) {
        const float4 t = *reinterpret_cast<const float4*>(b.p + e);
        y[e] = t.x;
        y[e + 1] = t.y;
        y[e + 2] = t.z;
        y[e + 3] = t.w;
    }
    return widen_cost(cost_sqrt(sumsq8<DIM>(a.v, y)));
}

// Out rows of a sweep (its window of split rows), nout rows of Q columns:
// element (m, q) lives at ((q / C) * nout + m) * C + q % C, C the accumulators in
// 16 bytes.  The rows of one column chunk are consecutive, so a lane of the sweep
// stores its rows of a column block from one address with constant offsets; with
// nout = 1 this is the plain row.
template <typename Acc>
__host__ __device__ constexpr int out_chunk() {
    return 16 / (int)sizeof(Acc);
}
template <typename Acc>
__host__ __device__ __forceinline__ long long out_index(int m, int q, int nout) {
    constexpr int C = out_chunk<Acc>();
    return ((long long)(q / C) * nout + m) * C + q % C;
}

// Out-row number of frame row p of a sweep (window t, row e of it: t*owin + e),
// or -1 where p holds no split row.
__host__ __device__ __forceinline__ int out_row_of(const Sweep& s, int p) {
    if (s.nout <= 0) return -1;
    const int d = p - s.out_row0;
    if (d < 0) return -1;
    const int t = d / s.ospace, e = d - t * s.ospace;
    return (t < s.onw && e < s.owin) ? t * s.owin + e : -1;
}
// Frame row of out row m of a sweep.
__host__ __device__ __forceinline__ int out_frame_row(const Sweep& s, int m) {
    const int t = m / s.owin;
    return s.out_row0 + t * s.ospace + (m - t * s.owin);
}
// Whether frame rows [lo, hi) hold a split row of the sweep.
__host__ __device__ __forceinline__ bool out_rows_meet(const Sweep& s, int lo, int hi) {
    if (s.nout <= 0) return false;
    const int a = max(lo - s.out_row0, 0);
    const int t = a / s.ospace;
    if (t >= s.onw) return false;
    // the first window that ends after a: window t if a lies in it, else t + 1
    const int w = (a - t * s.ospace < s.owin) ? t : t + 1;
    return w < s.onw && s.out_row0 + w * s.ospace < hi;
}

// Cost of global cell (i, j) of a pair, for the split and checks.
template <int KIND, int DIM>
__device__ __forceinline__ auto cell_cost(const PairDesc& pd, int i, int j, int d) {
    Frame<KIND, DIM> a, b;
    a.load(pd.X, i, d);
    b.load(pd.Y, j, d);
    return frame_cost(a, b);
}

}  // namespace dtwb
