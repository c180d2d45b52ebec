/* Bipartite (two-sublattice) connected sums -- oracle body, included once per precision by
 * cos_oracle.c after oracle_impl.h.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call it.
 *
 * Setting (Methods A, bipartite lattices; Results A, sublattice-resolved masks; Alg. 1-2):
 * every interaction vertex i sits in a unit cell and carries an internal sublattice index
 * s_i in {A, B}, shared by its two density points (contact interaction).  The propagator
 * between points depends on both indices, a^l(i s_i, j s_j) = G^l_{s_i s_j}(X_i - X_j), and
 * a shift point at vertex i in a loop of flavor l carries sigma_{l, s_i} (the equal-time
 * shift (alpha +- Delta) / U differs between the sublattices).  The connected sum is summed
 * over every sublattice assignment (Methods A, strategy (i)):
 *     c_bip(V) = sum_{s in {A,B}^n} c(V; s),
 * c(V; s) the connected sum of the matrices M_s^l[i][j] = a^l(i s_i, j s_j) with per-vertex
 * shift weights sigma_{l, s_i}.
 *
 * Layouts: M4 = [l][i][s][j][t] (flavor, vertex, sublattice, vertex, sublattice), s, t in
 * {0 = A, 1 = B}; sig2 = [l][s] or NULL.
 */

/* c_bip by its definition: the sum over the 2^n assignments of one of the single-assignment
 * routes (method 0: merged DP, 1: determinants + subset subtraction, 2: brute force over
 * decorated covers of the tiled point matrix). */
int FN(bip_sum)(int n, int nf, int wt, const double *M4, const double *sig2, int absmode, int method,
                double *out_hi, double *out_lo) {
    if (n < 1 || n > 12 || nf < 1 || nf > 8 || wt < 1) return -1;
    if (method == 2 && (n > 5 || wt != 1 || absmode)) return -1;
    if (method == 1 && (wt != 1 || absmode)) return -1;
    const int np = 2 * n;
    double *Ms = (double *)malloc(sizeof(double) * nf * n * n);
    double *A = (double *)malloc(sizeof(double) * nf * np * np);
    double sv[8 * 12];
    REAL total = 0;
    for (unsigned s = 0; s < (1u << n); s++) {
        for (int l = 0; l < nf; l++)
            for (int i = 0; i < n; i++)
                for (int j = 0; j < n; j++) {
                    const int si = (s >> i) & 1, sj = (s >> j) & 1;
                    Ms[((size_t)l * n + i) * n + j] = M4[((((size_t)l * n + i) * 2 + si) * n + j) * 2 + sj];
                }
        if (sig2)
            for (int l = 0; l < nf; l++)
                for (int i = 0; i < n; i++) sv[l * n + i] = sig2[l * 2 + ((s >> i) & 1)];
        double hi = 0, lo = 0;
        int rc;
        if (method == 0) {
            rc = FN(dp_v)(n, nf, wt, Ms, sig2 ? sv : NULL, absmode, &hi, &lo);
        } else if (method == 1) {
            rc = FN(closed_v)(n, nf, Ms, sig2 ? sv : NULL, &hi, &lo, NULL, NULL);
        } else {
            /* point p sits at vertex p mod n: tile each flavor's matrix 2 x 2 */
            for (int l = 0; l < nf; l++)
                for (int p = 0; p < np; p++)
                    for (int q = 0; q < np; q++)
                        A[((size_t)l * np + p) * np + q] = Ms[((size_t)l * n + p % n) * n + q % n];
            rc = FN(brute_v)(n, nf, A, sig2 ? sv : NULL, 1, &hi, &lo);
        }
        if (rc) {
            free(Ms);
            free(A);
            return -1;
        }
        total += (REAL)hi + (REAL)lo;
    }
    *out_hi = (double)total;
    *out_lo = (double)(total - (REAL)(*out_hi));
    free(Ms);
    free(A);
    return 0;
}

/* The sublattice-resolved merged DP (Results A; Alg. 1-2 with the contact merge), in plain
 * push loops.  Interaction mask digits d_i: 0 untouched, 1 half-visited on A, 2 half-visited
 * on B, 3 full (the sublattice of a full vertex is forgotten).  State (mu, h, s_h, v, s_v, l):
 * mu as a base-4 code, the open loop's head vertex h with its sublattice, the current
 * endpoint v with its sublattice, the loop's flavor l.
 *  - start: the loop through the normal point of vertex 0 on sublattice s, weight 1; if
 *    vertex 0 carries a shift point, weight -2 sigma_{l,s} at mu_0 = full.
 *  - extend to j with d_j != 3: d_j = 0 -> for both s_j: weight 2 a^l(v s_v, j s_j), and with
 *    shifts also the full j with weight 2 a^l(v s_v, j s_j) (-sigma_{l,s_j}); d_j half ->
 *    s_j from the mask, weight a^l(v s_v, j s_j), j becomes full.
 *  - close: C(mu) += -w a^l(v s_v, h s_h) (times the loop weight wt); a half-visited vertex k
 *    (smallest index) opens the next loop at its other point on its recorded sublattice:
 *    (mu with k full, k, s_k, k, s_k, l') += C(mu) for every flavor l'; the full mask feeds
 *    the sink; otherwise the cover is disconnected and dropped.
 * Memory: three layers of C(2n, ell) codes x (2n)^2 x nf values (n <= 8). */
int FN(bip_dp4)(int n, int nf, int wt, const double *M4_in, const double *sig2_in, int absmode,
                double *out_hi, double *out_lo) {
    if (n < 1 || n > 8 || nf < 1 || nf > 8 || wt < 1) return -1;
    int p4[10];
    p4[0] = 1;
    for (int i = 1; i <= n; i++) p4[i] = 4 * p4[i - 1];
    const int ncode = p4[n];
    const size_t msz = (size_t)nf * n * 2 * n * 2;
    REAL *M = (REAL *)malloc(sizeof(REAL) * msz);
    for (size_t k = 0; k < msz; k++) M[k] = absmode ? RABS((REAL)M4_in[k]) : (REAL)M4_in[k];
    REAL sig[8 * 2];
    int shifts = 0;
    for (int k = 0; k < nf * 2; k++) {
        sig[k] = sig2_in ? (REAL)sig2_in[k] : 0;
        if (absmode) sig[k] = RABS(sig[k]);
        if (sig[k] != 0) shifts = 1;
    }
    const REAL sgn = absmode ? 1 : -1;
    static const int wdig[4] = {0, 1, 1, 2};
    int *layer = (int *)malloc(sizeof(int) * ncode);
    int *rank = (int *)malloc(sizeof(int) * ncode);
    int cnt[25] = {0};
    for (int code = 0; code < ncode; code++) {
        int x = code, s = 0;
        for (int i = 0; i < n; i++) { s += wdig[x % 4]; x /= 4; }
        layer[code] = s;
        rank[code] = cnt[s]++;
    }
    const size_t blk = (size_t)n * 2 * n * 2 * nf;   /* (h, s_h, v, s_v, l) block of one mask */
    size_t maxcnt = 0;
    for (int s = 0; s <= 2 * n; s++) if ((size_t)cnt[s] > maxcnt) maxcnt = cnt[s];
    REAL *ring[3];
    for (int r = 0; r < 3; r++) ring[r] = (REAL *)calloc(maxcnt * blk, sizeof(REAL));
    REAL *C = (REAL *)malloc(sizeof(REAL) * maxcnt);
#define ST(code, h, sh, v, sv, l) \
    ring[layer[code] % 3][(size_t)rank[code] * blk + ((((size_t)(h) * 2 + (sh)) * n + (v)) * 2 + (sv)) * nf + (l)]
#define A4(l, v, sv, j, sj) M[((((size_t)(l) * n + (v)) * 2 + (sv)) * n + (j)) * 2 + (sj)]
    for (int s0 = 0; s0 < 2; s0++)
        for (int l = 0; l < nf; l++) {
            ST(1 + s0, 0, s0, 0, s0, l) += 1;                                  /* mu_0 = half on s0 */
            if (shifts) ST(3, 0, s0, 0, s0, l) += sgn * 2 * sig[l * 2 + s0];   /* mu_0 = full */
        }
    REAL S = 0;
    for (int ell = 1; ell <= 2 * n; ell++) {
        for (int code = 0; code < ncode; code++) {
            if (layer[code] != ell || code % 4 == 0) continue;
            int d[8], x = code;
            for (int i = 0; i < n; i++) { d[i] = x % 4; x /= 4; }
            REAL Cmu = 0;
            for (int h = 0; h < n; h++)
                for (int sh = 0; sh < 2; sh++)
                    for (int v = 0; v < n; v++)
                        for (int sv = 0; sv < 2; sv++)
                            for (int l = 0; l < nf; l++) {
                                const REAL w = ST(code, h, sh, v, sv, l);
                                if (w == 0) continue;
                                Cmu += sgn * w * A4(l, v, sv, h, sh) * wt;
                                for (int j = 0; j < n; j++) {
                                    if (d[j] == 3) continue;
                                    if (d[j] == 0) {
                                        for (int sj = 0; sj < 2; sj++) {
                                            const REAL e = w * 2 * A4(l, v, sv, j, sj);
                                            ST(code + (1 + sj) * p4[j], h, sh, j, sj, l) += e;
                                            if (shifts) ST(code + 3 * p4[j], h, sh, j, sj, l) += e * (sgn * sig[l * 2 + sj]);
                                        }
                                    } else {
                                        const int sj = d[j] - 1;
                                        ST(code + (3 - d[j]) * p4[j], h, sh, j, sj, l) += w * A4(l, v, sv, j, sj);
                                    }
                                }
                            }
            C[rank[code]] = Cmu;
        }
        for (int code = 0; code < ncode; code++) {
            if (layer[code] != ell || code % 4 == 0) continue;
            int k = -1, full = 1, dk = 0, x = code;
            for (int i = 0; i < n; i++) {
                const int dd = x % 4;
                x /= 4;
                if ((dd == 1 || dd == 2) && k < 0) { k = i; dk = dd; }
                if (dd != 3) full = 0;
            }
            if (k >= 0) {
                const int sk = dk - 1;
                for (int l = 0; l < nf; l++) ST(code + (3 - dk) * p4[k], k, sk, k, sk, l) += C[rank[code]];
            } else if (full) {
                S += C[rank[code]];
            }
        }
        memset(ring[ell % 3], 0, maxcnt * blk * sizeof(REAL));
    }
#undef ST
#undef A4
    *out_hi = (double)S;
    *out_lo = (double)(S - (REAL)(*out_hi));
    for (int r = 0; r < 3; r++) free(ring[r]);
    free(C); free(layer); free(rank); free(M);
    return 0;
}
