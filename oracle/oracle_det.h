/* SU(2) connected sums with determinant weights -- oracle body, included once per precision
 * by cos_oracle.c after oracle_impl.h.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call it.
 *
 * Setting (Results A, the variant without cycle factors; Alg. 1): 2n points, point p < n is
 * the spin-up end of interaction vertex p and point p + n its spin-down end (the interaction
 * lines (i, i + n)).  The matrix is block diagonal in spin: a(p s, q t) = G_b(i s, j t) when
 * p = b n + i and q = b n + j lie in the same block b, and there is no edge between blocks.
 * With nsub = 2 every vertex carries a sublattice index s in {A, B} shared by its two points
 * and the sum runs over every assignment (Methods A, strategy (i)); nsub = 1 is the plain
 * lattice.  The sum of all diagrams of a vertex set S is a(S) = sum_s det(A_up[S; s])
 * det(A_dn[S; s]); the DP returns its connected part c(V).
 *
 * Alg. 1 as stated, in push form over layers of visited-point counts:
 *  - state ((u, s_u), (v, s_v), mu): head point u of the open clow, current point v (same spin
 *    block), interaction mask mu with digits 0 (unvisited), (1, s) (visited once, on
 *    sublattice s), 2 (visited twice; its sublattice is forgotten).  Only the interaction's
 *    visit count is kept, not which of its points was visited, so sequences that visit one
 *    point twice (nonphysical clows) are generated; they cancel in pairs.
 *  - start: u = v = point 0 on either sublattice, mask (1, s) at vertex 0, weight 1.
 *  - extend: to every point w of v's block other than the head u whose interaction is not
 *    full; an unvisited interaction is entered on either sublattice, a half-visited one on
 *    its recorded sublattice; weight a(v s_v, w s_w).
 *  - close: weight -a(v s_v, u s_u); the next clow opens at the smallest half-visited
 *    interaction k, at either of its two points except the current head, on k's recorded
 *    sublattice; with no half-visited interaction the sequence is disconnected and dropped.
 *  - sink: the states with every interaction full close once more into S.
 *
 * Layouts: G = [b][i][s][j][t] (spin block, vertex, sublattice, vertex, sublattice), alpha =
 * [b][s] or NULL: the diagonal a(p s, p s) carries - alpha_{b, s} (the shifted density of the
 * interaction (n_up - alpha_up)(n_dn - alpha_dn)).  absmode: |entries|, |alpha| added to the
 * diagonal and every sign +, an upper bound on the sum of |terms|.
 * Memory: two layers of (codes of the layer) x 2 (n nsub)^2 values: n <= 10 (nsub = 1) and
 * n <= 8 (nsub = 2). */
int FN(det_clow)(int n, int nsub, const double *G_in, const double *alpha_in, int absmode, double *out_hi,
                 double *out_lo) {
    if (n < 1 || nsub < 1 || nsub > 2 || (nsub == 1 && n > 10) || (nsub == 2 && n > 8)) return -1;
    const int base = nsub + 2, FULL = nsub + 1, ns = n * nsub;
    int pw[12];
    pw[0] = 1;
    for (int i = 1; i <= n; i++) pw[i] = base * pw[i - 1];
    const int ncode = pw[n];
    /* a(b; i s; j t) with the shifted diagonal */
    const size_t asz = (size_t)2 * ns * ns;
    REAL *a = (REAL *)malloc(sizeof(REAL) * asz);
    for (size_t k = 0; k < asz; k++) a[k] = absmode ? RABS((REAL)G_in[k]) : (REAL)G_in[k];
    if (alpha_in)
        for (int b = 0; b < 2; b++)
            for (int i = 0; i < n; i++)
                for (int s = 0; s < nsub; s++) {
                    const REAL al = (REAL)alpha_in[b * nsub + s];
                    a[((size_t)b * ns + i * nsub + s) * ns + i * nsub + s] += absmode ? RABS(al) : -al;
                }
#define AM(b, i, s, j, t) a[((size_t)(b) * ns + (i) * nsub + (s)) * ns + (j) * nsub + (t)]
    const REAL sgn = absmode ? 1 : -1;
    /* layer of a mask = number of visited points */
    int *layer = (int *)malloc(sizeof(int) * ncode);
    int *rank = (int *)malloc(sizeof(int) * ncode);
    int cnt[2 * 12 + 1] = {0};
    for (int code = 0; code < ncode; code++) {
        int x = code, l = 0;
        for (int i = 0; i < n; i++) {
            const int d = x % base;
            x /= base;
            l += d == 0 ? 0 : (d == FULL ? 2 : 1);
        }
        layer[code] = l;
        rank[code] = cnt[l]++;
    }
    size_t maxcnt = 0;
    for (int l = 0; l <= 2 * n; l++)
        if ((size_t)cnt[l] > maxcnt) maxcnt = cnt[l];
    const size_t blk = (size_t)2 * ns * ns; /* (b, u = (i_u, s_u), v = (i_v, s_v)) of one mask */
    REAL *ring[2];
    for (int r = 0; r < 2; r++) ring[r] = (REAL *)calloc(maxcnt * blk, sizeof(REAL));
#define ST(code, b, iu, su, iv, sv) \
    ring[layer[code] % 2][(size_t)rank[code] * blk + (((size_t)(b) * ns + (iu) * nsub + (su)) * ns + (iv) * nsub + (sv))]
    for (int s = 0; s < nsub; s++) ST((1 + s) * pw[0], 0, 0, s, 0, s) = 1;
    REAL S = 0;
    for (int ell = 1; ell <= 2 * n; ell++) {
        memset(ring[(ell + 1) % 2], 0, maxcnt * blk * sizeof(REAL));
        for (int code = 0; code < ncode; code++) {
            if (layer[code] != ell) continue;
            int d[12], x = code, k = -1;
            for (int i = 0; i < n; i++) {
                d[i] = x % base;
                x /= base;
                if (k < 0 && d[i] >= 1 && d[i] <= nsub) k = i;
            }
            for (int b = 0; b < 2; b++)
                for (int iu = 0; iu < n; iu++)
                    for (int su = 0; su < nsub; su++)
                        for (int iv = 0; iv < n; iv++)
                            for (int sv = 0; sv < nsub; sv++) {
                                const REAL w = ST(code, b, iu, su, iv, sv);
                                if (w == 0) continue;
                                const REAL cl = sgn * w * AM(b, iv, sv, iu, su);
                                if (ell == 2 * n) { /* sink */
                                    S += cl;
                                    continue;
                                }
                                /* extend within block b, never onto the head point */
                                for (int j = 0; j < n; j++) {
                                    if (j == iu || d[j] == FULL) continue;
                                    if (d[j] == 0) {
                                        for (int sj = 0; sj < nsub; sj++)
                                            ST(code + (1 + sj) * pw[j], b, iu, su, j, sj) += w * AM(b, iv, sv, j, sj);
                                    } else {
                                        const int sj = d[j] - 1;
                                        ST(code + (FULL - d[j]) * pw[j], b, iu, su, j, sj) += w * AM(b, iv, sv, j, sj);
                                    }
                                }
                                /* close; open at either point of k except the head */
                                if (k >= 0) {
                                    const int sk = d[k] - 1;
                                    for (int bh = 0; bh < 2; bh++) {
                                        if (bh == b && k == iu) continue;
                                        ST(code + (FULL - d[k]) * pw[k], bh, k, sk, k, sk) += cl;
                                    }
                                }
                            }
        }
    }
#undef ST
#undef AM
    *out_hi = (double)S;
    *out_lo = (double)(S - (REAL)(*out_hi));
    for (int r = 0; r < 2; r++) free(ring[r]);
    free(layer);
    free(rank);
    free(a);
    return 0;
}
