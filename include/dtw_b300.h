/*
 * dtw_b300.h -- C ABI of the B300 (sm_103a) exact linear-memory DTW alignment
 * library (Tralie & Dempsey, "Exact, Parallelizable Dynamic Time Warping
 * Alignment with Linear Memory").
 *
 * Problem (Section 2.1): X holds M frames and Y holds N frames of dimension d.
 * A warping path is a list of K index pairs starting at (0,0), ending at
 * (M-1,N-1), each step adding (0,1), (1,0) or (1,1).  Its cost is the sum of the
 * frame costs C(i,j) over its pairs; DTW finds a path of minimum cost D*.
 * Frame costs: Euclidean distance of FP32 frames (Section 4.1) or |x - y| of
 * int32 samples (d must be 1).
 *
 * The library computes D* and an optimal path with the divide-and-conquer
 * recursion of Section 3.2 (Algorithm 2): at each level every box of the level
 * is swept by a tiled wavefront (Algorithm 1's anti-diagonal order, Section 3.1)
 * that keeps only O(M+N) boundary state, a split row fixes one path cell per box
 * (Lemmas 1 and 2), and boxes below a size cutoff finish with a full-table DP
 * and backtrace (Section 2.1).
 *
 * Tie rule: the returned path is the path a textbook backtrace yields when each
 * backpointer is the first minimum in the order DIAG (i-1,j-1), UP (i-1,j),
 * LEFT (i,j-1).  For DTW_ABS_I32 the result is exact (int accumulation) and the
 * path is that canonical path bit for bit.  For DTW_EUCLID_F32 the frame cost
 * is evaluated in FP32 and accumulated in FP64; the cost is within 1e-6
 * relative of the FP64 optimum and the path is optimal within that tolerance
 * (another path of equal cost may be returned).
 *
 * Memory: the caller owns X, Y, the path buffers and every output.  The library
 * owns a device workspace of dtw_footprint() bytes that grows on demand
 * (cudaMalloc) unless the caller provides an arena with dtw_set_arena().
 *
 * Pointers: X, Y and path_out may be host or device pointers; the library
 * detects which (cudaPointerGetAttributes) and stages host buffers through its
 * workspace.  All work runs on the stream set with dtw_set_stream() (default:
 * the legacy default stream) on the current device.
 *
 * Errors: every call returns a status (negative on error, see dtw_status); no
 * call aborts the process or throws.  The library is not re-entrant: calls
 * from several host threads are serialised by an internal lock.
 */
#ifndef DTW_B300_H
#define DTW_B300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DTW_API __attribute__((visibility("default")))
#else
#define DTW_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Frame cost kinds: the low byte of cost_kind. */
enum dtw_kind {
    DTW_EUCLID_F32 = 0, /* sqrt(sum_k (x_k - y_k)^2) of FP32 frames; FP64 accumulation */
    DTW_ABS_I32 = 1,    /* |x - y| of int32 samples (d == 1); exact int accumulation */
    /* Weighted edit distance of int32 symbol sequences (d == 1), which Section 5
     * names as a problem of the same dynamic-programming design, aligned by the
     * same linear-memory recursion.  Nodes (a, b), 0 <= a <= M, 0 <= b <= N,
     * stand for a symbols of X and b of Y aligned; E(0,0) = 0 and
     *   E(a,b) = min(E(a-1,b-1) + s, E(a-1,b) + gap, E(a,b-1) + gap)
     * with s = 0 for X[a-1] == Y[b-1], else sub (DTW_OPT_EDIT_SUB and
     * DTW_OPT_EDIT_GAP, default 1 and 1: Levenshtein distance).  The path is the
     * node sequence from (0,0) to (M,N) (K <= M+N+1 pairs; path_out capacity
     * 2*(M+N+1) int32), canonical under the tie order DIAG, UP, LEFT; the cost
     * is exact.  Symbols may not be INT32_MIN (used as a sentinel); the call
     * fails with DTW_EOVERFLOW unless (M+N+2) * max(sub, gap) < 2^29.  No form
     * flags; dtw_submit and dtw_cost_noalloc do not take this kind. */
    DTW_EDIT_I32 = 2
};

/* Form flags, OR-ed into cost_kind. */
enum dtw_form {
    /* The paper's own GPU design (Algorithm 1 inside Algorithm 2): one kernel
     * launch per anti-diagonal, one thread per cell, three rotating diagonal
     * buffers, FP64 cost and accumulation, recursion on the host, textbook DTW
     * when a box side drops below 500 (Section 3.2).  It is the comparator the
     * tiled path is measured against; its path is optimal but, under ties, not
     * necessarily the canonical one. */
    DTW_PLAIN_F64 = 1 << 8,
    /* With DTW_EUCLID_F32: the accumulated costs are compensated FP32 pairs
     * (hi + lo, about 48 significant bits; each FP32 frame cost added with
     * TwoSum) instead of FP64 values, which keeps the DP off the narrow FP64
     * pipe.  The split comparison still runs in FP64.  The cost matches the FP64
     * form to about 1e-9 relative on the bundled workloads (the FP32 frame
     * costs, shared by both forms, carry the 1e-7 error). */
    DTW_DP_F32_KAHAN = 1 << 10,
    /* With DTW_EUCLID_F32 and d == 64: a reduced-precision form.  The frame cost
     * is the expanded form sqrt(max(0, |x|^2 + |y|^2 - 2 x.y)) with the squared
     * norms in FP32 and the dot product of the BF16-rounded frames on the tensor
     * cores (FP32 accumulation) in 32 x 32 cost tiles; the DP is the
     * compensated FP32 one (implies DTW_DP_F32_KAHAN).  Its error against the
     * exact FP64 optimum is far above 1e-6: BF16 keeps 8 significant bits and the
     * expanded form cancels where frames are close, i.e. along the optimal path
     * (the measured error on the 60000 x 75000 MFCC-like pair is stated in the
     * library's design notes).  The returned path is a warping path; its cost is
     * the optimum of the form's own costs. */
    DTW_COST_BF16 = 1 << 9
};

enum dtw_status {
    DTW_OK = 0,
    DTW_PENDING = 1,    /* dtw_poll: the request has not finished */
    DTW_EINVAL = -1,    /* bad argument (null pointer, M or N < 1, d mismatch, unknown kind) */
    DTW_ENOMEM = -2,    /* workspace allocation failed or exceeds the budget */
    DTW_ECUDA = -3,     /* a CUDA runtime call failed */
    DTW_ETIMEOUT = -4,  /* a device-side wait exceeded its bound; the call was abandoned */
    DTW_EOVERFLOW = -5, /* max|x-y| * (M+N-1) does not fit the exact integer accumulator */
    DTW_EBUSY = -6,     /* the serving queue is full */
    DTW_EINTERNAL = -7  /* a device-side consistency check failed (a library bug) */
};

/*
 * dtw_align -- exact DTW cost and optimal warping path of one pair.
 *   X        M*d row-major frames (float for DTW_EUCLID_F32, int32 for DTW_ABS_I32)
 *   Y        N*d row-major frames of the same type
 *   d        feature dimension (1 for DTW_ABS_I32)
 *   path_out capacity 2*(M+N-1) int32; receives K (i,j) pairs, (0,0) first
 *            (DTW_EDIT_I32: 2*(M+N+1), K nodes (a,b) from (0,0) to (M,N))
 *   cost_out host double; receives D* (exact integer value for DTW_ABS_I32
 *            and DTW_EDIT_I32)
 * Returns K (the path length, max(M,N) <= K <= M+N-1; for DTW_EDIT_I32
 * max(M,N)+1 <= K <= M+N+1) or a negative dtw_status.
 * Blocks until the result is in path_out and *cost_out.
 */
DTW_API int64_t dtw_align(const void* X, int64_t M, const void* Y, int64_t N, int32_t d,
                  int32_t cost_kind, int32_t* path_out, double* cost_out);

/*
 * dtw_cost -- D* only: one forward sweep of the whole accumulated-cost matrix
 * (Section 3.1), O(M+N) memory, no path.  Same arguments as dtw_align.
 * Returns DTW_OK or a negative dtw_status.
 */
DTW_API int dtw_cost(const void* X, int64_t M, const void* Y, int64_t N, int32_t d, int32_t cost_kind,
             double* cost_out);

/*
 * dtw_align_batch -- B independent pairs of uneven lengths, all aligned
 * together: every pair's boxes of a recursion level go out in the same kernel
 * launches.  X[b], Y[b], path_out[b] as in dtw_align (path_out[b] capacity
 * 2*(M[b]+N[b]-1) int32); K_out[b] and cost_out[b] receive path length and D*.
 * All pairs share d and cost_kind.  Returns DTW_OK or a negative dtw_status
 * (which then applies to the whole batch).
 */
DTW_API int dtw_align_batch(int32_t B, const void* const* X, const int64_t* M, const void* const* Y,
                    const int64_t* N, int32_t d, int32_t cost_kind, int32_t* const* path_out,
                    int64_t* K_out, double* cost_out);

/* One request of the asynchronous interface. */
typedef struct dtw_request {
    const void* X;
    int64_t M;
    const void* Y;
    int64_t N;
    int32_t d;
    int32_t cost_kind;
    int32_t* path_out; /* capacity 2*(M+N-1) int32, host or device */
} dtw_request;

/*
 * dtw_submit -- queue one alignment.  Returns a ticket >= 0 or a negative
 * dtw_status.  The request's buffers must stay valid until dtw_poll() for the
 * ticket returns something other than DTW_PENDING.
 * dtw_poll -- DTW_PENDING while running; DTW_OK once *K_out and *cost_out hold
 * the result (the ticket is then released); or a negative dtw_status.
 */
DTW_API int64_t dtw_submit(const dtw_request* r);
DTW_API int dtw_poll(int64_t ticket, int64_t* K_out, double* cost_out);

/* Stream for all subsequent work (a cudaStream_t; NULL = legacy default). */
DTW_API int dtw_set_stream(void* cuda_stream);

/* Device-memory budget for admission (0 = unlimited).  A call whose
 * dtw_footprint() exceeds it fails with DTW_ENOMEM before touching the GPU. */
DTW_API int dtw_set_budget(uint64_t bytes);

/* Caller-provided device arena (256-byte aligned) used instead of cudaMalloc for
 * the workspace; NULL releases it.  The arena must outlive every call made while
 * it is set. */
DTW_API int dtw_set_arena(void* device_ptr, uint64_t bytes);

/* Workspace bytes dtw_align needs for one pair; linear in M+N (Section 4.3's
 * memory argument): features staged from the host, per-level boundary rows,
 * box lists and the path. */
DTW_API size_t dtw_footprint(int64_t M, int64_t N, int32_t d, int32_t cost_kind);

DTW_API const char* dtw_strerror(int status);

/*
 * dtw_local_align -- local alignment (Smith-Waterman; Section 5 names it beside
 * edit distance as a problem of the same dynamic-programming design) of two
 * int32 symbol sequences, in linear memory on the same kernels.  Scores: +match
 * for equal symbols, -mismatch otherwise, -gap per gap (each 0 .. 2^20);
 *   H(a,b) = max(0, H(a-1,b-1) + score, H(a-1,b) - gap, H(a,b-1) - gap)
 * over nodes (a, b) as in DTW_EDIT_I32, H = 0 on row 0 and column 0; the local
 * score is S = max H.  The alignment returned (S > 0) is canonical:
 *   end    the first node in row-major order with H = S;
 *   start  among the nodes from which a global alignment to the end scores S,
 *          the largest in row-major order (the shortest such alignment);
 *   path   the canonical global alignment between them (tie order DIAG, UP,
 *          LEFT, as for DTW_EDIT_I32), K nodes from the start to the end.
 * Three passes: a forward sweep with the local floor (score and end), a sweep
 * of the reversed box from the end (start), and the edit-distance recursion on
 * the substrings between them.
 *   X, Y       int32 symbols (host or device), none equal to INT32_MIN or
 *              INT32_MIN + 1 (sentinels)
 *   path_out   capacity 2*(M+N+1) int32 (host or device); K (a,b) pairs
 *   K_out      host; the path length (0 when S = 0)
 *   score_out  host; S
 *   se_out     host, 4 int64: start a, start b, end a, end b (zeros when S = 0)
 * Returns DTW_OK, DTW_EINVAL, DTW_EOVERFLOW ((M+N+2) * max(match, mismatch, gap)
 * must stay below 2^29), DTW_ENOMEM, DTW_ECUDA or DTW_ETIMEOUT.  Blocks.
 */
DTW_API int dtw_local_align(const int32_t* X, int64_t M, const int32_t* Y, int64_t N, int32_t match,
                            int32_t mismatch, int32_t gap, int32_t* path_out, int64_t* K_out, int64_t* score_out,
                            int64_t* se_out);

/*
 * dtw_path_discrepancy -- the alignment discrepancy of two warping paths of the
 * same M x N problem (Section 4.3, Results): for every cell (i, j) of path 1,
 * its row error min |j - k| over the cells (i, k) of path 2 and its column error
 * min |i - k| over the cells (k, j) of path 2.  Used to compare the paths of two
 * precision forms, or a path that took another tie than the oracle's.
 *   P1, P2     K1 x 2 / K2 x 2 int32 (i, j) pairs, row-major, each a warping path
 *              from (0, 0) to (M-1, N-1) with steps (0,1), (1,0), (1,1); host or
 *              device pointers; max(M, N) <= K <= M + N - 1
 *   err_out    2*K1 int32, host or device: the row errors of P1's cells in path
 *              order, then their column errors
 *   max_out    host int32, the largest error (NULL: not wanted)
 * The caller owns every buffer.  Returns DTW_OK; DTW_EINVAL for bad sizes or a
 * path that is not a warping path of M x N (checked on the device; err_out is
 * then unspecified); DTW_ENOMEM or DTW_ECUDA.  Blocks until the result is
 * written.
 */
DTW_API int dtw_path_discrepancy(const int32_t* P1, int64_t K1, const int32_t* P2, int64_t K2, int64_t M, int64_t N,
                                 int32_t* err_out, int32_t* max_out);

/*
 * dtw_cost_noalloc -- D* of one pair, like dtw_cost, without allocating any
 * device memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc -- a process whose device memory is fully
 * reserved up front (a serving loop, a host application that owns the memory
 * budget of plug-ins it loads), or code that must not risk the implicit device
 * synchronisation and the latency of an allocation in the middle of its work.
 *
 * All scratch state lives in one fixed device array inside the library (about
 * 4.2 MB), which every GPU that loads the library keeps until the process
 * exits.  Limits: min(M, N) <= DTW_NOALLOC_MAX_SHORT and max(M, N) <=
 * DTW_NOALLOC_MAX_LONG; larger inputs are rejected with DTW_ENOMEM.
 *   X, Y       DEVICE pointers (host pointers are rejected with DTW_EINVAL)
 *   cost_kind  DTW_EUCLID_F32 or DTW_ABS_I32 (no form flags)
 *   cost_out   host double; receives D*
 *   cuda_stream  stream for the work (a cudaStream_t; NULL = legacy default)
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  Every call
 * reuses the same array and clears what has to start from zero; calls whose GPU
 * work overlaps (several streams or several threads at once) race on it, so
 * calls from several host threads are serialised and callers must not run two
 * on different streams concurrently.  Blocks until *cost_out is written.
 */
#define DTW_NOALLOC_MAX_SHORT 262144
#define DTW_NOALLOC_MAX_LONG 4194304
DTW_API int dtw_cost_noalloc(const void* X, int64_t M, const void* Y, int64_t N, int32_t d, int32_t cost_kind,
                             double* cost_out, void* cuda_stream);

/* Counters of the most recent dtw_align / dtw_cost / dtw_align_batch call. */
typedef struct dtw_stats {
    int64_t problem_cells;   /* sum of M*N over the pairs */
    int64_t sweep_cells;     /* cells evaluated by wavefront sweeps */
    int64_t tag_cells;       /* of which carried a split tag (integer kind) */
    int64_t base_cells;      /* cells evaluated by full-table base cases */
    int32_t levels;          /* recursion levels swept */
    int32_t sweep_launches;  /* sweep kernel launches */
    int32_t base_boxes;      /* boxes finished by the base-case kernel */
    int32_t kernel_launches; /* CUDA kernels the call launched */
    int32_t retagged_boxes;  /* integer boxes whose split window tied and were re-swept with tags */
    int32_t pad;
    int64_t resyncs;         /* boundary prefetch refills (a band waited for the band above) */
    int64_t polls;           /* failed polls of boundary words while waiting */
    double sweep_ms;         /* summed device time of the sweep launches (timing on) */
    double device_ms;        /* device time of the whole call (timing on) */
} dtw_stats;

DTW_API int dtw_get_stats(dtw_stats* out);

/*
 * dtw_pipe_rates -- measured issue rates of the instructions that the per-cell
 * roofline counts (the cell update of the recurrence, Section 2.1): for each, the
 * whole device's thread-instruction rate per second, timed alone at full
 * occupancy with eight independent chains per thread on the current device:
 *   [0] three-way signed 32-bit minimum (__vimin3_s32; the chains also issue one
 *       XOR per eight minima, so this is a lower bound)
 *   [1] 32-bit sum of absolute difference (__sad: |x - y| + z)
 *   [2] FP32 fused multiply-add
 *   [3] packed FP32x2 fused multiply-add (one instruction, two lanes of work)
 *   [4] correctly rounded FP32 square root (__fsqrt_rn; several instructions)
 *   [5] FP64 add
 * and then, measured by one warp running a single chain of 2048 operations that
 * each take the previous one's result (clock64 cycles per operation), the
 * latencies that set the pace of a recurrence's dependency chain:
 *   [6] __vimin3_s32   [7] __sad   [8] FP32 add   [9] FP64 add
 *   [10] a warp shuffle (__shfl_up_sync by one lane)
 *   rates_out  host, n doubles; entries past the eleventh are not written
 * Returns the number of entries written, DTW_EINVAL (NULL or n < 1), DTW_ENOMEM
 * or DTW_ECUDA.  Allocates and frees a small device buffer and a stream of its
 * own; blocks for some tens of milliseconds.
 */
DTW_API int dtw_pipe_rates(double* rates_out, int32_t n);

/* Tuning and instrumentation switches (dtw_set_option keys). */
enum dtw_option {
    DTW_OPT_TIMING = 1,      /* 1: record CUDA events around each launch (default 0) */
    DTW_OPT_BASE_AREA = 2,   /* boxes of at most this many cells finish in the base case */
    DTW_OPT_SPIN_LIMIT = 3,  /* polls before a device-side wait gives up (DTW_ETIMEOUT) */
    DTW_OPT_SKIP_PUBLISH = 4, /* test hook: one band never publishes (exercises DTW_ETIMEOUT) */
    DTW_OPT_GRAPH = 5,        /* 1 (default): the level loop of dtw_align / dtw_align_batch runs as one CUDA
                                 graph with a device-side loop condition (no host round trip per level);
                                 0: a host loop that reads the control block back after every level.
                                 DTW_OPT_TIMING on forces the host loop (it times every level). */
    DTW_OPT_SWEEP_VARIANT = 6, /* integer-kind sweep lane block: 0 (default) 4 rows x 4 columns per lane and
                                 step, 1: 2 x 4, 2: 8 x 4, 3: 4 x 4 with each 8-step group as straight-line
                                 code (faster on long bands) (chosen by the autotuner in the Python package) */
    DTW_OPT_EDIT_SUB = 7,     /* DTW_EDIT_I32: cost of a substitution, 0 .. 2^20 (default 1) */
    DTW_OPT_EDIT_GAP = 8,     /* DTW_EDIT_I32: cost of an insertion or a deletion, 0 .. 2^20 (default 1) */
    DTW_OPT_NOALLOC_EPOCH = 9, /* test hook: the next dtw_cost_noalloc call starts its boundary-word epochs at
                                  this value, 0 .. 2^32-1 (exercises the restart near the 32-bit limit) */
    DTW_OPT_FUSED_SPLIT = 10, /* where dtw_align / dtw_align_batch run each level's split (the argmin of
                                 F + B - C, Lemma 2): 1 (default) in the sweep kernel, whose blocks take split
                                 items once the sweep tickets are gone, for float kinds and for batches of
                                 two or more pairs, and in a separate launch for a single integer or edit
                                 pair (measured faster for it); 2 always in the sweep kernel; 0 always in a
                                 separate launch.  The BF16 cost form always uses the separate launch.
                                 Results are the same in every case. */
    DTW_OPT_SPLIT_WINDOWS = 11 /* windows of split rows per box and recursion level, at most: 1 .. 15
                                 (default 7).  Lemma 1 holds for any row that every warping path crosses,
                                 so each box's forward and backward sweeps may end on several equally
                                 spaced split rows (windows of 9 rows for the integer and edit kinds, one
                                 row for the others) and each window fixes one cell of the optimal path
                                 (Lemma 2): the box splits into up to that many + 1 pieces.  1 is the
                                 paper's single middle split.  Fewer levels and a shorter dependency
                                 chain per alignment for about the same work (2MN cells); the window
                                 count shrinks on boxes too small for it.  Integer and edit paths are
                                 the same for every value; float costs agree within rounding.  Takes
                                 effect for serving engines started afterwards. */
};
DTW_API int dtw_set_option(int32_t key, int64_t value);

#ifdef __cplusplus
}
#endif

#endif /* DTW_B300_H */
