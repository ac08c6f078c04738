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

/* Diagonal step into node (a, b): cost CM for equal symbols, else S (CM is 0
 * for edit distance; the local-alignment oracle below uses a negative CM). */
static int64_t sub_cost(const int32_t *X, const int32_t *Y, int64_t a, int64_t b, int64_t CM, int64_t S) {
    return X[a - 1] == Y[b - 1] ? CM : S;
}

/* E over the whole node grid, row by row; ptr (if not NULL) gets one pointer per
 * node.  E is (M+1) x (N+1), row-major. */
static void edit_table_cm(const int32_t *X, int64_t M, const int32_t *Y, int64_t N, int64_t CM, int64_t S, int64_t G,
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
                const int64_t dg = E[(a - 1) * W + b - 1] + sub_cost(X, Y, a, b, CM, S);
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

static void edit_table(const int32_t *X, int64_t M, const int32_t *Y, int64_t N, int64_t S, int64_t G, int64_t *E,
                       uint8_t *ptr) {
    edit_table_cm(X, M, Y, N, 0, S, G, E, ptr);
}

/* The optimal cost and the canonical path (node pairs from (0,0) to (M,N);
 * path_out holds 2*(M+N+1) int32), with match cost CM (0 for edit distance). */
static int edit_align_cm(const int32_t *X, int64_t M, const int32_t *Y, int64_t N, int64_t CM, int64_t S, int64_t G,
                         int32_t *path_out, int64_t *K_out, int64_t *cost_out) {
    const int64_t W = N + 1, cells = (M + 1) * W;
    int64_t *E = (int64_t *)malloc((size_t)cells * sizeof(int64_t));
    uint8_t *ptr = (uint8_t *)malloc((size_t)cells);
    if (!E || !ptr) {
        free(E);
        free(ptr);
        return EO_ENOMEM;
    }
    edit_table_cm(X, M, Y, N, CM, S, G, E, ptr);
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

int oracle_edit(const int32_t *X, int64_t M, const int32_t *Y, int64_t N, int64_t S, int64_t G,
                int32_t *path_out, int64_t *K_out, int64_t *cost_out) {
    if (!X || !Y || M < 1 || N < 1 || S < 0 || G < 0 || M > INT32_MAX || N > INT32_MAX) return EO_EINVAL;
    return edit_align_cm(X, M, Y, N, 0, S, G, path_out, K_out, cost_out);
}

/*
 * Local alignment (Smith-Waterman; Section 5 names it beside edit distance):
 * scores +MA for a match, -MM for a mismatch, -G for a gap;
 *   H(a, b) = max(0, H(a-1,b-1) + sigma, H(a-1,b) - G, H(a,b-1) - G), H = 0 on
 *   row 0 and column 0; the optimal local score is S = max H.
 * The alignment returned (S > 0):
 *   end   e = (a_e, b_e), the first node in row-major order with H = S;
 *   start s = (a_s, b_s), among the nodes from which a global alignment to e
 *           scores S, the largest in row-major order (the shortest alignment);
 *   path  the canonical global alignment from s to e (the edit-distance rules
 *         with costs -MA, MM, G and the tie order DIAG, UP, LEFT).
 * se_out gets a_s, b_s, a_e, b_e.  With S = 0 the path is empty (K = 0).
 */
int oracle_local(const int32_t *X, int64_t M, const int32_t *Y, int64_t N, int64_t MA, int64_t MM, int64_t G,
                 int32_t *path_out, int64_t *K_out, int64_t *score_out, int64_t *se_out) {
    if (!X || !Y || M < 1 || N < 1 || MA < 0 || MM < 0 || G < 0 || M > INT32_MAX || N > INT32_MAX) return EO_EINVAL;
    const int64_t W = N + 1, cells = (M + 1) * W;
    int64_t *H = (int64_t *)malloc((size_t)cells * sizeof(int64_t));
    if (!H) return EO_ENOMEM;
    int64_t best = 0, ae = 0, be = 0;
    for (int64_t a = 0; a <= M; ++a) {
        for (int64_t b = 0; b <= N; ++b) {
            int64_t v = 0;
            if (a > 0 && b > 0) {
                const int64_t dg = H[(a - 1) * W + b - 1] + (X[a - 1] == Y[b - 1] ? MA : -MM);
                const int64_t up = H[(a - 1) * W + b] - G;
                const int64_t lf = H[a * W + b - 1] - G;
                if (dg > v) v = dg;
                if (up > v) v = up;
                if (lf > v) v = lf;
            }
            H[a * W + b] = v;
            if (v > best) {  /* strictly greater: the first node in row-major order */
                best = v;
                ae = a;
                be = b;
            }
        }
    }
    *score_out = best;
    if (best == 0) {
        free(H);
        *K_out = 0;
        return EO_OK;
    }
    /* R(a, b): the best global-alignment score from node (a, b) to e */
    const int64_t Wr = be + 1;
    int64_t *R = H; /* reuse: (ae+1) x (be+1) <= cells */
    int64_t as = -1, bs = -1;
    for (int64_t a = ae; a >= 0; --a) {
        for (int64_t b = be; b >= 0; --b) {
            int64_t v;
            if (a == ae && b == be) {
                v = 0;
            } else {
                v = INT64_MIN / 4;
                if (a < ae && b < be) {
                    const int64_t dg = R[(a + 1) * Wr + b + 1] + (X[a] == Y[b] ? MA : -MM);
                    if (dg > v) v = dg;
                }
                if (a < ae && R[(a + 1) * Wr + b] - G > v) v = R[(a + 1) * Wr + b] - G;
                if (b < be && R[a * Wr + b + 1] - G > v) v = R[a * Wr + b + 1] - G;
            }
            R[a * Wr + b] = v;
            if (as < 0 && v == best) { /* the first hit scanning backwards: the largest node */
                as = a;
                bs = b;
            }
        }
    }
    free(H);
    if (as < 0) return EO_EINVAL; /* cannot happen: some start reaches S */
    int64_t cost = 0;
    int rc = edit_align_cm(X + as, ae - as, Y + bs, be - bs, -MA, MM, G, path_out, K_out, &cost);
    if (rc) return rc;
    for (int64_t t = 0; t < *K_out; ++t) {
        path_out[2 * t] += (int32_t)as;
        path_out[2 * t + 1] += (int32_t)bs;
    }
    se_out[0] = as;
    se_out[1] = bs;
    se_out[2] = ae;
    se_out[3] = be;
    return -cost == best ? EO_OK : EO_EINVAL;
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
