/*
 * Oracle bodies, instantiated by dtw_oracle.c once per accumulation type.
 * Expects ACC (accumulator type), ACC_INF (a value larger than any reachable
 * cost), SFX (symbol suffix) and COSTFN (the frame cost C(i,j)) to be defined.
 * TEST INFRASTRUCTURE ONLY.
 */
#define OR_CAT2(a, b) a##b
#define OR_CAT(a, b) OR_CAT2(a, b)
#define FN(name) OR_CAT(name, SFX)

/* Oracle 1 on the box [i0, i0+Ms) x [j0, j0+Ns): textbook DTW (Section 2.1).
 * D(0,j) and D(i,0) are prefix sums of C along the first row and column
 * (Eq. "dtwboundary"); every other cell is min(LEFT, UP, DIAG) + C (Eq.
 * "recurrence").  The backpointer P(i,j) is the first strict minimum in the
 * order DIAG, UP, LEFT; the backtrace follows P from the last cell to the first.
 * Appends the box's path, first cell first, to l. */
static int FN(textbook)(const prob_t *p, int64_t i0, int64_t j0, int64_t Ms, int64_t Ns,
                        plist_t *l, ACC *cost) {
    uint8_t *P = (uint8_t *)calloc((size_t)((Ms * Ns + 3) / 4), 1);
    ACC *prev = (ACC *)malloc((size_t)Ns * sizeof(ACC));
    ACC *cur = (ACC *)malloc((size_t)Ns * sizeof(ACC));
    if (!P || !prev || !cur) {
        free(P);
        free(prev);
        free(cur);
        return OR_ENOMEM;
    }
#define SETP(a, b, v) (P[((a) * Ns + (b)) >> 2] |= (uint8_t)((v) << ((((a) * Ns + (b)) & 3) * 2)))
#define GETP(a, b) ((P[((a) * Ns + (b)) >> 2] >> ((((a) * Ns + (b)) & 3) * 2)) & 3)
    for (int64_t a = 0; a < Ms; ++a) {
        for (int64_t b = 0; b < Ns; ++b) {
            ACC c = COSTFN(p, i0 + a, j0 + b);
            ACC best;
            int mv;
            if (a == 0 && b == 0) {
                best = 0;
                mv = MV_NONE;
            } else if (a == 0) {
                best = cur[b - 1];
                mv = MV_LEFT;
            } else if (b == 0) {
                best = prev[0];
                mv = MV_UP;
            } else {
                ACC dg = prev[b - 1], up = prev[b], lf = cur[b - 1];
                best = dg;
                mv = MV_DIAG;
                if (up < best) {
                    best = up;
                    mv = MV_UP;
                }
                if (lf < best) {
                    best = lf;
                    mv = MV_LEFT;
                }
            }
            cur[b] = best + c;
            SETP(a, b, mv);
        }
        ACC *t = prev;
        prev = cur;
        cur = t;
    }
    *cost = prev[Ns - 1];
    /* backtrace from (Ms-1, Ns-1) to (0, 0), then append in forward order */
    int64_t start = l->n, a = Ms - 1, b = Ns - 1;
    int rc = OR_OK;
    for (;;) {
        rc = plist_push(l, i0 + a, j0 + b);
        if (rc) break;
        int mv = (int)GETP(a, b);
        if (mv == MV_NONE) break;
        if (mv == MV_DIAG) {
            --a;
            --b;
        } else if (mv == MV_UP) {
            --a;
        } else {
            --b;
        }
    }
    if (rc == OR_OK) {
        for (int64_t x = start, y = l->n - 1; x < y; ++x, --y) {
            int32_t ti = l->v[2 * x], tj = l->v[2 * x + 1];
            l->v[2 * x] = l->v[2 * y];
            l->v[2 * x + 1] = l->v[2 * y + 1];
            l->v[2 * y] = ti;
            l->v[2 * y + 1] = tj;
        }
    }
#undef SETP
#undef GETP
    free(P);
    free(prev);
    free(cur);
    return rc;
}

/* Whole forward (reverse == 0) or backward (reverse != 0) accumulated-cost
 * matrix, written row-major into out.  The backward matrix is the forward one of
 * the reversed series read back in original coordinates (Section 3.2, Lemma 2). */
static int FN(accmat)(const prob_t *p, int32_t reverse, ACC *out) {
    const int64_t M = p->M, N = p->N;
    for (int64_t a = 0; a < M; ++a) {
        for (int64_t b = 0; b < N; ++b) {
            int64_t i = reverse ? M - 1 - a : a, j = reverse ? N - 1 - b : b;
            int64_t pi = reverse ? i + 1 : i - 1, pj = reverse ? j + 1 : j - 1;
            ACC c = COSTFN(p, i, j), best;
            if (a == 0 && b == 0)
                best = 0;
            else if (a == 0)
                best = out[i * N + pj];
            else if (b == 0)
                best = out[pi * N + j];
            else {
                ACC dg = out[pi * N + pj], up = out[pi * N + j], lf = out[i * N + pj];
                best = dg;
                if (up < best) best = up;
                if (lf < best) best = lf;
            }
            out[i * N + j] = best + c;
        }
    }
    return OR_OK;
}

/* Diagonal DTW (Algorithm 1) on the box [i0, i0+Ms) x [j0, j0+Ns), forward from
 * the box's first cell, or on the reversed box (rev != 0) from its last cell.
 * Local cell (a, b) lies on anti-diagonal a + b and maps to global (i0+a, j0+b),
 * or to (i0+Ms-1-a, j0+Ns-1-b) when reversed.  Diagonals 0..kstop are evaluated
 * in order, each from the two before it, in three circularly shifted buffers
 * indexed by a.  On return o0, o1, o2 hold diagonals kstop-2, kstop-1, kstop
 * (ACC_INF where a diagonal has no cell at that a).  Adds the number of cells
 * evaluated to *cells. */
static int FN(diagdtw)(const prob_t *p, int64_t i0, int64_t j0, int64_t Ms, int64_t Ns, int rev,
                       int64_t kstop, ACC *o0, ACC *o1, ACC *o2, int64_t *cells) {
    ACC *buf = (ACC *)malloc((size_t)(3 * Ms) * sizeof(ACC));
    if (!buf) return OR_ENOMEM;
    ACC *dm2 = buf, *dm1 = buf + Ms, *dk = buf + 2 * Ms;
    for (int64_t a = 0; a < 3 * Ms; ++a) buf[a] = ACC_INF;
    for (int64_t k = 0; k <= kstop; ++k) {
        int64_t alo = k - (Ns - 1) > 0 ? k - (Ns - 1) : 0;
        int64_t ahi = k < Ms - 1 ? k : Ms - 1;
        for (int64_t a = 0; a < Ms; ++a) dk[a] = ACC_INF;
        for (int64_t a = alo; a <= ahi; ++a) {
            int64_t b = k - a;
            int64_t gi = rev ? i0 + Ms - 1 - a : i0 + a;
            int64_t gj = rev ? j0 + Ns - 1 - b : j0 + b;
            ACC c = COSTFN(p, gi, gj), best;
            if (k == 0) {
                best = 0;
            } else {
                best = ACC_INF;
                if (a >= 1 && b >= 1 && dm2[a - 1] < best) best = dm2[a - 1]; /* DIAG (a-1,b-1) */
                if (a >= 1 && dm1[a - 1] < best) best = dm1[a - 1];          /* UP   (a-1,b)   */
                if (b >= 1 && dm1[a] < best) best = dm1[a];                  /* LEFT (a,b-1)   */
            }
            dk[a] = best + c;
        }
        if (ahi >= alo) *cells += ahi - alo + 1;
        ACC *t = dm2; /* circular shift: k becomes k-1, k-1 becomes k-2 */
        dm2 = dm1;
        dm1 = dk;
        dk = t;
    }
    /* after the last shift dk still holds diagonal kstop-2 */
    memcpy(o0, dk, (size_t)Ms * sizeof(ACC));
    memcpy(o1, dm2, (size_t)Ms * sizeof(ACC));
    memcpy(o2, dm1, (size_t)Ms * sizeof(ACC));
    free(buf);
    return OR_OK;
}

/* Oracle 2: Algorithm 2 on the box [i0, i0+Ms) x [j0, j0+Ns).  Appends the box's
 * path to l (first cell first) and counts evaluated cells. */
static int FN(linmdtw)(const prob_t *p, int64_t i0, int64_t j0, int64_t Ms, int64_t Ns, int64_t m,
                       plist_t *l, int64_t *cells) {
    /* base case (Algorithm 2's recursion stop); a side of 1 or 2 always stops,
     * since such a box can have a child equal to itself */
    if (Ms < m || Ns < m || Ms <= 2 || Ns <= 2) {
        ACC c;
        *cells += Ms * Ns;
        return FN(textbook)(p, i0, j0, Ms, Ns, l, &c);
    }
    const int64_t K = Ms + Ns - 1;     /* number of anti-diagonals */
    const int64_t cd = (K - 1) / 2;    /* the split set is diagonals cd-1, cd, cd+1 */
    const int64_t kf = cd + 1;         /* forward stop: ceil(K/2) in 1-based counting */
    const int64_t kb = K - 1 - (cd - 1); /* backward stop, one more than kf when K is even */
    ACC *w = (ACC *)malloc((size_t)(6 * Ms) * sizeof(ACC));
    if (!w) return OR_ENOMEM;
    ACC *f0 = w, *f1 = w + Ms, *f2 = w + 2 * Ms, *b0 = w + 3 * Ms, *b1 = w + 4 * Ms, *b2 = w + 5 * Ms;
    int rc = FN(diagdtw)(p, i0, j0, Ms, Ns, 0, kf, f0, f1, f2, cells);
    if (rc == OR_OK) rc = FN(diagdtw)(p, i0, j0, Ms, Ns, 1, kb, b0, b1, b2, cells);
    int64_t pa = -1, pb = -1;
    if (rc == OR_OK) {
        /* forward diagonal cd-1+t pairs with reversed diagonal kb-t, i.e.
         * (f0,b2), (f1,b1), (f2,b0); a cell at local row a sits at reversed row
         * Ms-1-a.  S = F + B - C (Lemma 2); pivot = argmin, ties to the lowest
         * diagonal, then to the lowest row. */
        ACC *fd[3] = {f0, f1, f2}, *bd[3] = {b2, b1, b0};
        ACC best = ACC_INF;
        for (int t = 0; t < 3; ++t) {
            int64_t k = cd - 1 + t;
            int64_t alo = k - (Ns - 1) > 0 ? k - (Ns - 1) : 0;
            int64_t ahi = k < Ms - 1 ? k : Ms - 1;
            for (int64_t a = alo; a <= ahi; ++a) {
                int64_t bb = k - a;
                ACC S = fd[t][a] + bd[t][Ms - 1 - a] - COSTFN(p, i0 + a, j0 + bb);
                if (S < best) {
                    best = S;
                    pa = a;
                    pb = bb;
                }
            }
        }
    }
    free(w);
    if (rc) return rc;
    /* recurse on the two boxes that share the pivot; drop the repeated pivot */
    rc = FN(linmdtw)(p, i0, j0, pa + 1, pb + 1, m, l, cells);
    if (rc) return rc;
    l->n--;
    return FN(linmdtw)(p, i0 + pa, j0 + pb, Ms - pa, Ns - pb, m, l, cells);
}

#undef FN
#undef OR_CAT
#undef OR_CAT2
