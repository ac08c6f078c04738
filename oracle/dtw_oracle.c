/*
 * CPU oracle for exact DTW alignment -- TEST INFRASTRUCTURE, not product code.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code, header, table or helper with the CUDA
 * path and includes nothing from it.  It is deliberately plain and slow.
 *
 * Two oracles, each instantiated twice from oracle_impl.h (FP64 accumulation
 * for Euclidean costs of FP32 features, int64 accumulation for |x-y| costs of
 * int32 samples):
 *
 *   oracle 1  textbook DTW (Section 2.1): the accumulated-cost recurrence
 *             (Eq. "recurrence") with its boundary rows (Eq. "dtwboundary"),
 *             a backpointer per cell and a backtrace.  The backpointer is the
 *             first strict minimum in the order DIAG, UP, LEFT, where UP is
 *             (i-1, j) and LEFT is (i, j-1) as in Eq. "recurrence".
 *   oracle 2  the divide-and-conquer linear-memory alignment (Algorithm 2,
 *             Section 3.2) in the paper's geometry: a diagonal sweep
 *             (Algorithm 1) forward and one on the reversed series, the
 *             split cost F + B - C (Lemma 2) on three central anti-diagonals
 *             (Lemma 1), argmin pivot, recursion, textbook DTW on boxes with a
 *             side below m.  It also counts processed cells (Section 3.2).
 *
 * Floating-point rules: every cost is sqrt(sum_k (x_k - y_k)^2) evaluated in
 * double, k ascending, no fused multiply-add (the file is compiled with
 * -ffp-contract=off); an accumulated cost is "min of the predecessors, then
 * + C(i,j)".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_EUCLID_F32 = 0, OR_ABS_I32 = 1 };
enum { MV_DIAG = 0, MV_UP = 1, MV_LEFT = 2, MV_NONE = 3 };
enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2 };

typedef struct {
    const void *X, *Y;
    int64_t M, N;
    int32_t d;
} prob_t;

/* Frame cost C_{X,Y}(i,j) (Section 2.1); Euclidean distance per Section 4.1. */
static double cost_euclid(const prob_t *p, int64_t i, int64_t j) {
    const float *x = (const float *)p->X + i * p->d;
    const float *y = (const float *)p->Y + j * p->d;
    double s = 0.0;
    for (int k = 0; k < p->d; ++k) {
        double t = (double)x[k] - (double)y[k];
        s = s + t * t;
    }
    return sqrt(s);
}

static int64_t cost_absdiff(const prob_t *p, int64_t i, int64_t j) {
    int64_t t = (int64_t)((const int32_t *)p->X)[i] - (int64_t)((const int32_t *)p->Y)[j];
    return t < 0 ? -t : t;
}

/* growable list of (i, j) pairs */
typedef struct {
    int32_t *v;
    int64_t n, cap;
} plist_t;

static int plist_push(plist_t *l, int64_t i, int64_t j) {
    if (l->n == l->cap) {
        int64_t nc = l->cap ? 2 * l->cap : 256;
        int32_t *nv = (int32_t *)realloc(l->v, (size_t)nc * 2 * sizeof(int32_t));
        if (!nv) return OR_ENOMEM;
        l->v = nv;
        l->cap = nc;
    }
    l->v[2 * l->n] = (int32_t)i;
    l->v[2 * l->n + 1] = (int32_t)j;
    l->n++;
    return OR_OK;
}

#define ACC double
#define ACC_INF (INFINITY)
#define SFX _f64
#define COSTFN cost_euclid
#include "oracle_impl.h"
#undef ACC
#undef ACC_INF
#undef SFX
#undef COSTFN

#define ACC int64_t
#define ACC_INF (INT64_MAX / 4)
#define SFX _i64
#define COSTFN cost_absdiff
#include "oracle_impl.h"
#undef ACC
#undef ACC_INF
#undef SFX
#undef COSTFN

/* A frame cost given as an explicit M x N matrix (row-major FP64, held in p->X;
 * p->Y and p->d unused): for a cost form evaluated outside the oracle, such as
 * the tensor-core form's expanded Euclidean cost (Section 4.1 with the frames
 * rounded to BF16).  Only the textbook DP and backtrace are used with it. */
static double cost_given(const prob_t *p, int64_t i, int64_t j) {
    return ((const double *)p->X)[i * p->N + j];
}

#pragma GCC diagnostic push
#pragma GCC diagnostic ignored "-Wunused-function"
#define ACC double
#define ACC_INF (INFINITY)
#define SFX _given
#define COSTFN cost_given
#include "oracle_impl.h"
#undef ACC
#undef ACC_INF
#undef SFX
#undef COSTFN
#pragma GCC diagnostic pop

static int check_args(const void *X, int64_t M, const void *Y, int64_t N, int32_t d, int32_t kind) {
    if (!X || !Y || M < 1 || N < 1 || d < 1) return OR_EINVAL;
    if (kind != OR_EUCLID_F32 && kind != OR_ABS_I32) return OR_EINVAL;
    if (kind == OR_ABS_I32 && d != 1) return OR_EINVAL;
    if (M > INT32_MAX || N > INT32_MAX) return OR_EINVAL;
    return OR_OK;
}

/* ---- exported entry points (double results are exact integers for OR_ABS_I32) ---- */

/* Oracle 1: textbook DTW.  path_out holds 2*(M+N-1) int32, filled from (0,0) to
 * (M-1,N-1); *K_out receives the path length. */
int oracle_dtw(const void *X, int64_t M, const void *Y, int64_t N, int32_t d, int32_t kind,
               int32_t *path_out, int64_t *K_out, double *cost_out, int64_t *icost_out) {
    int rc = check_args(X, M, Y, N, d, kind);
    if (rc) return rc;
    prob_t p = {X, Y, M, N, d};
    plist_t l = {0, 0, 0};
    if (kind == OR_EUCLID_F32) {
        double c = 0;
        rc = textbook_f64(&p, 0, 0, M, N, &l, &c);
        if (cost_out) *cost_out = c;
        if (icost_out) *icost_out = 0;
    } else {
        int64_t c = 0;
        rc = textbook_i64(&p, 0, 0, M, N, &l, &c);
        if (cost_out) *cost_out = (double)c;
        if (icost_out) *icost_out = c;
    }
    if (rc == OR_OK) {
        memcpy(path_out, l.v, (size_t)l.n * 2 * sizeof(int32_t));
        *K_out = l.n;
    }
    free(l.v);
    return rc;
}

/* Oracle 2: linmdtw (Algorithm 2) with base-case parameter m (>= 3).
 * *cells_out receives the number of accumulated-cost cells evaluated. */
int oracle_linmdtw(const void *X, int64_t M, const void *Y, int64_t N, int32_t d, int32_t kind,
                   int64_t m, int32_t *path_out, int64_t *K_out, double *cost_out,
                   int64_t *icost_out, int64_t *cells_out) {
    int rc = check_args(X, M, Y, N, d, kind);
    if (rc) return rc;
    if (m < 3) return OR_EINVAL;
    prob_t p = {X, Y, M, N, d};
    plist_t l = {0, 0, 0};
    int64_t cells = 0;
    if (kind == OR_EUCLID_F32) {
        rc = linmdtw_f64(&p, 0, 0, M, N, m, &l, &cells);
    } else {
        rc = linmdtw_i64(&p, 0, 0, M, N, m, &l, &cells);
    }
    if (rc == OR_OK) {
        memcpy(path_out, l.v, (size_t)l.n * 2 * sizeof(int32_t));
        *K_out = l.n;
        *cells_out = cells;
        /* the cost of the returned path, summed along it in path order */
        if (kind == OR_EUCLID_F32) {
            double s = 0;
            for (int64_t k = 0; k < l.n; ++k) s = s + cost_euclid(&p, l.v[2 * k], l.v[2 * k + 1]);
            if (cost_out) *cost_out = s;
            if (icost_out) *icost_out = 0;
        } else {
            int64_t s = 0;
            for (int64_t k = 0; k < l.n; ++k) s += cost_absdiff(&p, l.v[2 * k], l.v[2 * k + 1]);
            if (cost_out) *cost_out = (double)s;
            if (icost_out) *icost_out = s;
        }
    }
    free(l.v);
    return rc;
}

/* Full M x N matrix of the forward accumulated cost D (reverse == 0) or of the
 * backward cost B (reverse != 0): B(i,j) is the optimal cost of a warping path
 * from (i,j) to (M-1,N-1), C(i,j) included.  For small problems only. */
int oracle_acc_matrix(const void *X, int64_t M, const void *Y, int64_t N, int32_t d, int32_t kind,
                      int32_t reverse, double *out_f, int64_t *out_i) {
    int rc = check_args(X, M, Y, N, d, kind);
    if (rc) return rc;
    prob_t p = {X, Y, M, N, d};
    if (kind == OR_EUCLID_F32) return accmat_f64(&p, reverse, out_f);
    return accmat_i64(&p, reverse, out_i);
}

/* Sum of C along a given list of K (i,j) pairs. */
int oracle_path_cost(const void *X, int64_t M, const void *Y, int64_t N, int32_t d, int32_t kind,
                     const int32_t *path, int64_t K, double *cost_out, int64_t *icost_out) {
    int rc = check_args(X, M, Y, N, d, kind);
    if (rc) return rc;
    prob_t p = {X, Y, M, N, d};
    double s = 0;
    int64_t si = 0;
    for (int64_t k = 0; k < K; ++k) {
        int64_t i = path[2 * k], j = path[2 * k + 1];
        if (i < 0 || i >= M || j < 0 || j >= N) return OR_EINVAL;
        if (kind == OR_EUCLID_F32)
            s = s + cost_euclid(&p, i, j);
        else
            si += cost_absdiff(&p, i, j);
    }
    if (cost_out) *cost_out = kind == OR_EUCLID_F32 ? s : (double)si;
    if (icost_out) *icost_out = si;
    return OR_OK;
}

/* Oracle 1 on a given FP64 cost matrix C (M x N, row-major): the textbook DP,
 * backpointers (first strict minimum in the order DIAG, UP, LEFT) and backtrace
 * of Section 2.1, unchanged; only C(i,j) is read from the matrix. */
int oracle_dtw_given(const double *C, int64_t M, int64_t N, int32_t *path_out, int64_t *K_out, double *cost_out) {
    if (!C || M < 1 || N < 1 || M > INT32_MAX || N > INT32_MAX) return OR_EINVAL;
    prob_t p = {C, C, M, N, 1};
    plist_t l = {0, 0, 0};
    double c = 0;
    int rc = textbook_given(&p, 0, 0, M, N, &l, &c);
    if (rc == OR_OK) {
        memcpy(path_out, l.v, (size_t)l.n * 2 * sizeof(int32_t));
        *K_out = l.n;
        *cost_out = c;
    }
    free(l.v);
    return rc;
}
