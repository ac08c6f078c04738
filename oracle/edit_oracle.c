/*
 * CPU oracle for edit-distance alignment -- TEST INFRASTRUCTURE, not product code.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares nothing with the CUDA path.
 *
 * Section 5 names edit distance as a problem with the same dynamic-programming
 * design as DTW, one that the linear-memory recursion carries over to.  This is
 * its plain definition (weighted Levenshtein distance), written out with a
 * pointer per node and a backtrace:
 *
 *   nodes (a, b), 0 <= a <= M, 0 <= b <= N: a symbols of X and b of Y aligned;
 *   E(0, 0) = 0, E(a, 0) = a G, E(0, b) = b G;
 *   E(a, b) = min( E(a-1, b-1) + s(X[a-1], Y[b-1])   DIAG (match or substitute)
 *                  E(a-1, b)   + G                   UP   (X[a-1] against a gap)
 *                  E(a, b-1)   + G )                 LEFT (Y[b-1] against a gap)
 *   with s(x, y) = 0 if x == y, else S.
 *
 * The pointer is the first strict minimum in the order DIAG, UP, LEFT (the tie
 * order of the DTW oracle); row 0 has only LEFT, column 0 only UP.  The path is
 * the node sequence from (0, 0) to (M, N).  int64 throughout.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { EO_DIAG = 0, EO_UP = 1, EO_LEFT = 2, EO_NONE = 3 };
enum { EO_OK = 0, EO_EINVAL = -1, EO_ENOMEM = -2 };

static int64_t sub_cost(const int32_t *X, const int32_t *Y, int64_t a, int64_t b, int64_t S) {
    return X[a - 1] == Y[b - 1] ? 0 : S;
}

/* E over the whole node grid, row by row; ptr (if not NULL) gets one pointer per
 * node.  E is (M+1) x (N+1), row-major. */
static void edit_table(const int32_t *X, int64_t M, const int32_t *Y, int64_t N, int64_t S, int64_t G,
                       int64_t *E, uint8_t *ptr) {
    const int64_t W = N + 1;
    for (int64_t a = 0; a <= M; ++a) {
        for (int64_t b = 0; b <= N; ++b) {
            int64_t v;
            uint8_t pt;
            if (a == 0 && b == 0) {
                v = 0;
                pt = EO_NONE;
            } else if (a == 0) {
                v = E[b - 1] + G;
                pt = EO_LEFT;
            } else if (b == 0) {
                v = E[(a - 1) * W] + G;
                pt = EO_UP;
            } else {
                const int64_t dg = E[(a - 1) * W + b - 1] + sub_cost(X, Y, a, b, S);
                const int64_t up = E[(a - 1) * W + b] + G;
                const int64_t lf = E[a * W + b - 1] + G;
                v = dg;
                pt = EO_DIAG;
                if (up < v) {
                    v = up;
                    pt = EO_UP;
                }
                if (lf < v) {
                    v = lf;
                    pt = EO_LEFT;
                }
            }
            E[a * W + b] = v;
            if (ptr) ptr[a * W + b] = pt;
        }
    }
}

/* The optimal cost and the canonical path (node pairs from (0,0) to (M,N);
 * path_out holds 2*(M+N+1) int32). */
int oracle_edit(const int32_t *X, int64_t M, const int32_t *Y, int64_t N, int64_t S, int64_t G,
                int32_t *path_out, int64_t *K_out, int64_t *cost_out) {
    if (!X || !Y || M < 1 || N < 1 || S < 0 || G < 0 || M > INT32_MAX || N > INT32_MAX) return EO_EINVAL;
    const int64_t W = N + 1, cells = (M + 1) * W;
    int64_t *E = (int64_t *)malloc((size_t)cells * sizeof(int64_t));
    uint8_t *ptr = (uint8_t *)malloc((size_t)cells);
    if (!E || !ptr) {
        free(E);
        free(ptr);
        return EO_ENOMEM;
    }
    edit_table(X, M, Y, N, S, G, E, ptr);
    *cost_out = E[cells - 1];
    /* backtrace, then reverse into path_out */
    int64_t a = M, b = N, K = 0;
    for (;;) {
        path_out[2 * K] = (int32_t)a;
        path_out[2 * K + 1] = (int32_t)b;
        ++K;
        const uint8_t pt = ptr[a * W + b];
        if (pt == EO_NONE) break;
        if (pt == EO_DIAG) {
            --a;
            --b;
        } else if (pt == EO_UP) {
            --a;
        } else {
            --b;
        }
    }
    for (int64_t t = 0; t < K / 2; ++t) {
        int32_t ti = path_out[2 * t], tj = path_out[2 * t + 1];
        path_out[2 * t] = path_out[2 * (K - 1 - t)];
        path_out[2 * t + 1] = path_out[2 * (K - 1 - t) + 1];
        path_out[2 * (K - 1 - t)] = ti;
        path_out[2 * (K - 1 - t) + 1] = tj;
    }
    *K_out = K;
    free(E);
    free(ptr);
    return EO_OK;
}

/* The whole E table ((M+1) x (N+1) int64), and with reverse != 0 the table of the
 * reversed sequences (E_R(a, b): cost of aligning the last a symbols of X with
 * the last b of Y), for the split identity of the recursion. */
int oracle_edit_table(const int32_t *X, int64_t M, const int32_t *Y, int64_t N, int64_t S, int64_t G,
                      int32_t reverse, int64_t *out) {
    if (!X || !Y || M < 1 || N < 1 || S < 0 || G < 0) return EO_EINVAL;
    if (!reverse) {
        edit_table(X, M, Y, N, S, G, out, NULL);
        return EO_OK;
    }
    int32_t *XR = (int32_t *)malloc((size_t)M * sizeof(int32_t));
    int32_t *YR = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    if (!XR || !YR) {
        free(XR);
        free(YR);
        return EO_ENOMEM;
    }
    for (int64_t i = 0; i < M; ++i) XR[i] = X[M - 1 - i];
    for (int64_t j = 0; j < N; ++j) YR[j] = Y[N - 1 - j];
    edit_table(XR, M, YR, N, S, G, out, NULL);
    free(XR);
    free(YR);
    return EO_OK;
}
