/* Oracle implementation body, included once per precision by cos_oracle.c.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call it.
 *
 * Before inclusion the includer defines
 *   REAL    the arithmetic type (double, long double or __float128)
 *   FN(x)   the name of function x for this precision (a suffix is appended)
 *   RABS(x) absolute value in REAL
 *
 * Conventions (paper, Results A and Methods):
 *   - order n: n interaction vertices; vertex i carries two density points,
 *     i and i+n (the interaction lines I = {(i, i+n)} of Alg. 1-2).
 *   - M[l][i][j] (flavor l, vertices i, j) is the propagator G0^l(X_i - X_j);
 *     the 2n x 2n point matrix is M tiled 2 x 2 (Alg. 3 indexes A_l by
 *     vertex = point mod n).
 *   - a cover is a permutation of the points split into cycles; each closed
 *     cycle (fermion loop) carries a factor -1 and a flavor sum (Results A:
 *     sign (-1)^{n-k} for k cycles; flavor sum from the SU(N_f) discussion).
 *   - a shift point (counter-term, Methods A shifted action) replaces one
 *     point of a vertex; it carries -sigma_l, l the flavor of the loop through
 *     its partner (Alg. 3 Rule 2: a shift head inherits its partner's color and
 *     closes at once with sigma).  At most one shift point per vertex.
 */

/* ---------------------------------------------------------------- tier 0
 * Brute force over decorated covers (definition of the connected sum,
 * Results A: "sum over all connected Feynman diagrams"; cycle covers with
 * -1 and a flavor weight per closed loop).
 *
 * A      : nf point matrices, each (2n) x (2n), row-major; point p sits at
 *          vertex p mod n, its partner is (p + n) mod 2n.
 * sig    : nf shift weights, or NULL for no shift points.
 * connected: 1 = keep only covers whose vertex graph is connected
 *            (union-find over vertices, an edge p mod n -- pi(p) mod n for
 *            every normal point p); 0 = sum over all covers.
 * Cost: sum over decorations of (#normal points)!  -> n <= 5.
 */
typedef struct {
    int n, nf, np;        /* vertices, flavors, points = 2n */
    const REAL *A;        /* nf * np * np */
    const REAL *sig;      /* nf * n (flavor, vertex) or NULL */
    int connected;
    int is_shift[24];     /* point -> 1 if shift point */
    int normal[24];       /* list of normal points */
    int m;                /* number of normal points */
    int pi[24];           /* permutation image, indexed by point */
    REAL total;
} FN(brute_ctx);

static int FN(uf_find)(int *par, int x) {
    while (par[x] != x) x = par[x];
    return x;
}

static void FN(brute_leaf)(FN(brute_ctx) *c) {
    int n = c->n, np = c->np;
    if (c->connected) {
        int par[12];
        for (int i = 0; i < n; i++) par[i] = i;
        for (int a = 0; a < c->m; a++) {
            int p = c->normal[a];
            int r1 = FN(uf_find)(par, p % n), r2 = FN(uf_find)(par, c->pi[p] % n);
            if (r1 != r2) par[r1] = r2;
        }
        int root = FN(uf_find)(par, 0);
        for (int i = 1; i < n; i++)
            if (FN(uf_find)(par, i) != root) return;
    }
    int seen[24] = {0};
    REAL w = 1;
    for (int a = 0; a < c->m; a++) {
        int p0 = c->normal[a];
        if (seen[p0]) continue;
        /* collect the cycle through p0 */
        int cyc[24], len = 0, q = p0;
        while (!seen[q]) { seen[q] = 1; cyc[len++] = q; q = c->pi[q]; }
        REAL loop = 0;
        for (int l = 0; l < c->nf; l++) {
            const REAL *Al = c->A + (size_t)l * np * np;
            REAL t = 1;
            for (int e = 0; e < len; e++) t *= Al[cyc[e] * np + c->pi[cyc[e]]];
            if (c->sig) {
                for (int e = 0; e < len; e++) {
                    int partner = (cyc[e] + n) % np;
                    if (c->is_shift[partner]) t *= -c->sig[l * n + partner % n];
                }
            }
            loop += t;
        }
        w *= -loop;
    }
    c->total += w;
}

static void FN(brute_perm)(FN(brute_ctx) *c, int a, unsigned used) {
    if (a == c->m) { FN(brute_leaf)(c); return; }
    int p = c->normal[a];
    for (int b = 0; b < c->m; b++) {
        if (used & (1u << b)) continue;
        c->pi[p] = c->normal[b];
        FN(brute_perm)(c, a + 1, used | (1u << b));
    }
}

/* Sum over decorated covers, shift weights per (flavor, vertex): sig_in[l * n + i] is the
 * weight of a shift point at vertex i inside a loop of flavor l (a vertex-dependent shift,
 * e.g. the sublattice-dependent equal-time shift (alpha +- Delta) / U of Methods A).
 * Returns 0 on success, -1 on bad sizes. */
int FN(brute_v)(int n, int nf, const double *A_in, const double *sig_in, int connected,
                double *out_hi, double *out_lo) {
    if (n < 1 || n > 6 || nf < 1 || nf > 8) return -1;
    int np = 2 * n;
    REAL *A = (REAL *)malloc(sizeof(REAL) * nf * np * np);
    REAL sig[8 * 12];
    for (int k = 0; k < nf * np * np; k++) A[k] = (REAL)A_in[k];
    if (sig_in) for (int k = 0; k < nf * n; k++) sig[k] = (REAL)sig_in[k];
    REAL total = 0;
    int ndec = 1;
    for (int i = 0; i < n; i++) ndec *= sig_in ? 3 : 1;
    for (int d = 0; d < ndec; d++) {
        FN(brute_ctx) c;
        memset(&c, 0, sizeof c);
        c.n = n; c.nf = nf; c.np = np; c.A = A; c.sig = sig_in ? sig : NULL;
        c.connected = connected;
        /* decoration digit per vertex: 0 no shift, 1 point i is a shift,
           2 point i+n is a shift */
        int dd = d;
        for (int i = 0; i < n; i++) {
            int digit = dd % 3; dd /= 3;
            if (digit == 1) c.is_shift[i] = 1;
            if (digit == 2) c.is_shift[i + n] = 1;
        }
        c.m = 0;
        for (int p = 0; p < np; p++) if (!c.is_shift[p]) c.normal[c.m++] = p;
        c.total = 0;
        FN(brute_perm)(&c, 0, 0u);
        total += c.total;
    }
    *out_hi = (double)total;
    *out_lo = (double)(total - (REAL)(*out_hi));
    free(A);
    return 0;
}

/* Per-flavor shift weights (the same at every vertex). */
int FN(brute)(int n, int nf, const double *A_in, const double *sig_in, int connected,
              double *out_hi, double *out_lo) {
    if (n < 1 || n > 6 || nf < 1 || nf > 8) return -1;
    double sv[8 * 12];
    if (sig_in)
        for (int l = 0; l < nf; l++)
            for (int i = 0; i < n; i++) sv[l * n + i] = sig_in[l];
    return FN(brute_v)(n, nf, A_in, sig_in ? sv : NULL, connected, out_hi, out_lo);
}

/* ---------------------------------------------------------------- tier 1
 * Closed form from determinants and the subset subtraction of Methods A:
 *   c(S) = a(S) - sum_{T subset S, T != S, T contains min S} c(T) a(S \ T),
 * with a(empty) = 1 (reading: the sum of the paper's recursion excludes
 * S = V itself and fixes the block holding the smallest vertex).
 *
 * a(S), the sum over all decorated covers of the vertex set S, factorizes
 * over flavors once every point is given the flavor of its loop: a point set
 * of flavor l contributes (-1)^{size} det(M^l[.]) (sum over its
 * permutations with -1 per cycle), and a flavor holding both points of one
 * vertex has two equal rows, so vanishes.  Hence each vertex of S either
 * puts its two points in two different flavors (2 orderings), or has one
 * shift point (2 choices) and its normal point in flavor l (weight sigma_l;
 * the -1 of the shift and the sign of the missing point cancel).  Then
 *   a(S) = sum over such choices of prod sigma * prod_l det(M^l[J_l]),
 * J_l = vertices with a point in flavor l.  The sum over choices is taken
 * flavor by flavor with a per-vertex count c_v in {0,1,2} (base-3 code).
 * Cost ~ nf * 6^n.
 */
static REAL FN(det_sub)(int n, const REAL *M, unsigned J) {
    int idx[12], k = 0;
    for (int i = 0; i < n; i++) if (J & (1u << i)) idx[k++] = i;
    if (k == 0) return 1;
    REAL a[144];
    for (int r = 0; r < k; r++)
        for (int s = 0; s < k; s++) a[r * k + s] = M[idx[r] * n + idx[s]];
    REAL det = 1;
    for (int col = 0; col < k; col++) {
        int piv = col;
        REAL best = RABS(a[col * k + col]);
        for (int r = col + 1; r < k; r++)
            if (RABS(a[r * k + col]) > best) { best = RABS(a[r * k + col]); piv = r; }
        if (best == 0) return 0;
        if (piv != col) {
            for (int s = 0; s < k; s++) { REAL t = a[col * k + s]; a[col * k + s] = a[piv * k + s]; a[piv * k + s] = t; }
            det = -det;
        }
        REAL d = a[col * k + col];
        det *= d;
        for (int r = col + 1; r < k; r++) {
            REAL f = a[r * k + col] / d;
            for (int s = col; s < k; s++) a[r * k + s] -= f * a[col * k + s];
        }
    }
    return det;
}

/* a_out: 2^n values a(S) (may be NULL); c_out: 2^n values c(S) for S
 * containing vertex 0 (others 0; may be NULL).  Returns c(V). */
int FN(closed_v)(int n, int nf, const double *M_in, const double *sig_in,
                 double *out_hi, double *out_lo, double *a_out, double *c_out) {
    if (n < 1 || n > 12 || nf < 1 || nf > 8) return -1;
    int nsub = 1 << n;
    int p3[13];
    p3[0] = 1;
    for (int i = 1; i <= n; i++) p3[i] = 3 * p3[i - 1];
    REAL *M = (REAL *)malloc(sizeof(REAL) * nf * n * n);
    for (int k = 0; k < nf * n * n; k++) M[k] = (REAL)M_in[k];
    REAL sig[8 * 12];              /* [l][vertex] */
    int sig_any[8];
    for (int l = 0; l < nf; l++) {
        sig_any[l] = 0;
        for (int i = 0; i < n; i++) {
            sig[l * n + i] = sig_in ? (REAL)sig_in[l * n + i] : 0;
            if (sig[l * n + i] != 0) sig_any[l] = 1;
        }
    }
    REAL *det = (REAL *)malloc(sizeof(REAL) * nf * nsub);
    for (int l = 0; l < nf; l++)
        for (unsigned J = 0; J < (unsigned)nsub; J++) det[l * nsub + J] = FN(det_sub)(n, M + l * n * n, J);
    REAL *F = (REAL *)calloc(p3[n], sizeof(REAL));
    REAL *G = (REAL *)calloc(p3[n], sizeof(REAL));
    F[0] = 1;
    for (int l = 0; l < nf; l++) {
        memset(G, 0, sizeof(REAL) * p3[n]);
        for (int code = 0; code < p3[n]; code++) {
            if (F[code] == 0) continue;
            unsigned avail = 0, zeros = 0, ones = 0;
            int x = code;
            for (int v = 0; v < n; v++) {
                int cv = x % 3; x /= 3;
                if (cv < 2) avail |= 1u << v;
                if (cv == 0) zeros |= 1u << v;
                if (cv == 1) ones |= 1u << v;
            }
            /* every J subset of avail, including the empty set */
            unsigned J = avail;
            for (;;) {
                REAL d = det[l * nsub + J];
                if (d != 0) {
                    REAL w = d;
                    int c2 = code;
                    for (int v = 0; v < n; v++) if (J & (1u << v)) {
                        c2 += p3[v];
                        if (ones & (1u << v)) w *= 2;   /* second flavor of the vertex: 2 orderings */
                    }
                    G[c2] += F[code] * w;
                    /* shifted vertices among the untouched ones of J */
                    unsigned Z = J & zeros;
                    if (sig_in && sig_any[l] && Z) {
                        unsigned Sh = Z;
                        while (Sh) {
                            REAL ws = w;
                            int c3 = c2;
                            for (int v = 0; v < n; v++) if (Sh & (1u << v)) { ws *= 2 * sig[l * n + v]; c3 += p3[v]; }
                            G[c3] += F[code] * ws;
                            Sh = (Sh - 1) & Z;
                        }
                    }
                }
                if (J == 0) break;
                J = (J - 1) & avail;
            }
        }
        REAL *t = F; F = G; G = t;
    }
    REAL *a = (REAL *)malloc(sizeof(REAL) * nsub);
    for (unsigned S = 0; S < (unsigned)nsub; S++) {
        int code = 0;
        for (int v = 0; v < n; v++) if (S & (1u << v)) code += 2 * p3[v];
        a[S] = F[code];
    }
    REAL *c = (REAL *)calloc(nsub, sizeof(REAL));
    for (unsigned T = 1; T < (unsigned)nsub; T += 2) {    /* T contains vertex 0 */
        REAL acc = a[T];
        unsigned rest = T & ~1u;
        /* T' = {0} u R for every R strictly inside rest */
        for (unsigned R = (rest - 1) & rest;; R = (R - 1) & rest) {
            if (R == rest) break;
            unsigned Tp = R | 1u;
            acc -= c[Tp] * a[T & ~Tp];
            if (R == 0) break;
        }
        c[T] = acc;
    }
    REAL res = c[nsub - 1];
    *out_hi = (double)res;
    *out_lo = (double)(res - (REAL)(*out_hi));
    if (a_out) for (int S = 0; S < nsub; S++) a_out[S] = (double)a[S];
    if (c_out) for (int S = 0; S < nsub; S++) c_out[S] = (double)c[S];
    free(M); free(det); free(F); free(G); free(a); free(c);
    return 0;
}

int FN(closed)(int n, int nf, const double *M_in, const double *sig_in,
               double *out_hi, double *out_lo, double *a_out, double *c_out) {
    if (n < 1 || n > 12 || nf < 1 || nf > 8) return -1;
    double sv[8 * 12];
    if (sig_in)
        for (int l = 0; l < nf; l++)
            for (int i = 0; i < n; i++) sv[l * n + i] = sig_in[l];
    return FN(closed_v)(n, nf, M_in, sig_in ? sv : NULL, out_hi, out_lo, a_out, c_out);
}

/* ---------------------------------------------------------------- tier 2
 * The merged (contact-interaction) form of the cycle-aware DP of Results A
 * and Alg. 2-3, written as plain push loops in the paper's order.
 *
 * State (mu, h, v, l): mu_i in {0,1,2} counts the visited points of vertex i
 * (the interaction mask of Results A, which replaces the visited set R once
 * the two points of a vertex are merged), h the head vertex of the open loop,
 * v the vertex of its current point, l the loop's flavor (Alg. 3 heads carry
 * a flavor; continuing keeps it).
 *  - start: the loop through the normal point of vertex 0, weight 1; if
 *    vertex 0 carries a shift point (2 choices of which), weight -2 sigma_l.
 *  - extend (Alg. 2 Extend, Alg. 3 Rule 1): to an unvisited point at vertex j,
 *    weight M^l[v][j] times the number of such points (2 if mu_j = 0, 1 if
 *    mu_j = 1); entering an untouched vertex whose other point is a shift
 *    adds weight 2 M^l[v][j] (-sigma_l) and sets mu_j = 2 (Alg. 3: the shift
 *    takes its partner's color).
 *  - close (Alg. 2 Close, Alg. 3 Rule 2): C(mu) += -w M^l[v][h] (times the
 *    loop weight `wt` of a symmetric SU(N) run, Alg. 2 multiplies by N_f).
 *    A new loop opens at the unvisited point of the smallest half-visited
 *    vertex k (Results A: the new head has a visited partner, chosen by
 *    minimum index), in every flavor: (mu + e_k, k, k, l') += C(mu).  With
 *    every mu_i = 2, C(mu) goes to the sink; with none at 1 but some at 0 the
 *    cover is disconnected and is dropped.
 * absmode = 1 runs the same recursion on |M|, |sigma| with every sign +,
 * which bounds the sum of |term| (the "mass").
 */
int FN(dp_v)(int n, int nf, int wt, const double *M_in, const double *sig_in, int absmode,
             double *out_hi, double *out_lo) {
    if (n < 1 || n > 12 || nf < 1 || nf > 8 || wt < 1) return -1;
    int p3[14];
    p3[0] = 1;
    for (int i = 1; i <= n + 1; i++) p3[i] = 3 * p3[i - 1];
    int ncode = p3[n];
    REAL *M = (REAL *)malloc(sizeof(REAL) * nf * n * n);
    for (int k = 0; k < nf * n * n; k++) M[k] = absmode ? RABS((REAL)M_in[k]) : (REAL)M_in[k];
    REAL sig[8 * 12];              /* [l][vertex]: shift weight of vertex i in a loop of flavor l */
    int shifts = 0;
    for (int k = 0; k < nf * n; k++) {
        sig[k] = sig_in ? (REAL)sig_in[k] : 0;
        if (absmode) sig[k] = RABS(sig[k]);
        if (sig[k] != 0) shifts = 1;
    }
    REAL sgn = absmode ? 1 : -1;
    /* per-code layer and rank within the layer (layer = number of visited points) */
    int *layer = (int *)malloc(sizeof(int) * ncode);
    int *rank = (int *)malloc(sizeof(int) * ncode);
    int cnt[25] = {0};
    for (int code = 0; code < ncode; code++) {
        int x = code, s = 0;
        for (int i = 0; i < n; i++) { s += x % 3; x /= 3; }
        layer[code] = s;
        rank[code] = cnt[s]++;
    }
    size_t blk = (size_t)n * n * nf;   /* (h, v, l) block of one mask */
    REAL *ring[3];
    size_t maxcnt = 0;
    for (int s = 0; s <= 2 * n; s++) if ((size_t)cnt[s] > maxcnt) maxcnt = cnt[s];
    for (int r = 0; r < 3; r++) ring[r] = (REAL *)calloc(maxcnt * blk, sizeof(REAL));
    REAL *C = (REAL *)malloc(sizeof(REAL) * maxcnt);
#define ST(code, h, v, l) ring[layer[code] % 3][(size_t)rank[code] * blk + ((size_t)(h) * n + (v)) * nf + (l)]
    for (int l = 0; l < nf; l++) {
        ST(1, 0, 0, l) += 1;                                   /* mu = e_0 */
        if (shifts) ST(2, 0, 0, l) += sgn * 2 * sig[l * n];    /* mu = 2 e_0 */
    }
    REAL S = 0;
    for (int ell = 1; ell <= 2 * n; ell++) {
        for (int code = 0; code < ncode; code++) {
            if (layer[code] != ell || code % 3 == 0) continue;
            int mu[12], x = code;
            for (int i = 0; i < n; i++) { mu[i] = x % 3; x /= 3; }
            REAL Cmu = 0;
            for (int h = 0; h < n; h++)
                for (int v = 0; v < n; v++)
                    for (int l = 0; l < nf; l++) {
                        REAL w = ST(code, h, v, l);
                        if (w == 0) continue;
                        const REAL *Ml = M + (size_t)l * n * n;
                        Cmu += sgn * w * Ml[v * n + h] * wt;
                        for (int j = 0; j < n; j++) {
                            if (mu[j] == 2) continue;
                            ST(code + p3[j], h, j, l) += w * (mu[j] == 0 ? 2 : 1) * Ml[v * n + j];
                            if (mu[j] == 0 && shifts)
                                ST(code + 2 * p3[j], h, j, l) += w * 2 * Ml[v * n + j] * (sgn * sig[l * n + j]);
                        }
                    }
            C[rank[code]] = Cmu;
        }
        for (int code = 0; code < ncode; code++) {
            if (layer[code] != ell || code % 3 == 0) continue;
            int k = -1, full = 1, x = code;
            for (int i = 0; i < n; i++) {
                int d = x % 3; x /= 3;
                if (d == 1 && k < 0) k = i;
                if (d != 2) full = 0;
            }
            if (k >= 0) {
                for (int l = 0; l < nf; l++) ST(code + p3[k], k, k, l) += C[rank[code]];
            } else if (full) {
                S += C[rank[code]];
            }
        }
        /* layer ell is consumed: clear its ring slot for layer ell + 3 */
        memset(ring[ell % 3], 0, maxcnt * blk * sizeof(REAL));
    }
#undef ST
    *out_hi = (double)S;
    *out_lo = (double)(S - (REAL)(*out_hi));
    for (int r = 0; r < 3; r++) free(ring[r]);
    free(C); free(layer); free(rank); free(M);
    return 0;
}

/* Per-flavor shift weights (the same at every vertex). */
int FN(dp)(int n, int nf, int wt, const double *M_in, const double *sig_in, int absmode,
           double *out_hi, double *out_lo) {
    if (n < 1 || n > 12 || nf < 1 || nf > 8 || wt < 1) return -1;
    double sv[8 * 12];
    if (sig_in)
        for (int l = 0; l < nf; l++)
            for (int i = 0; i < n; i++) sv[l * n + i] = sig_in[l];
    return FN(dp_v)(n, nf, wt, M_in, sig_in ? sv : NULL, absmode, out_hi, out_lo);
}

/* Batch of configurations of one order (matrices packed [cfg][l][n][n]);
 * OpenMP over configurations.  Returns the number of threads used. */
int FN(dp_batch)(int n_cfg, int n, int nf, int wt, const double *M_in, const double *sig_in,
                 int absmode, double *out_hi, double *out_lo, int nthreads) {
    int used = 1;
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 1)
        for (int c = 0; c < n_cfg; c++) {
            double lo = 0;
            if (FN(dp)(n, nf, wt, M_in + (size_t)c * nf * n * n, sig_in, absmode, &out_hi[c], out_lo ? &out_lo[c] : &lo))
                err = 1;
        }
    }
#else
    (void)nthreads;
    for (int c = 0; c < n_cfg; c++) {
        double lo = 0;
        if (FN(dp)(n, nf, wt, M_in + (size_t)c * nf * n * n, sig_in, absmode, &out_hi[c], out_lo ? &out_lo[c] : &lo))
            err = 1;
    }
#endif
    return err ? -1 : used;
}
