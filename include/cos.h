/*
 * libcos -- connected-sum hot path of CoS++ (arXiv 2507.12349) on one B300.
 *
 * For each Monte Carlo configuration of n interaction vertices X_i = (r_i, tau_i)
 * the library returns the sum of all connected Feynman diagrams of order n of a
 * square-lattice SU(N_f) Hubbard model (Methods A: "the coefficients f_n are
 * the sum of all connected diagrams at order n"), evaluated with the
 * cycle-aware clow-sequence dynamic program of Results A and Alg. 2-3, in its
 * merged contact-interaction form (Results A: interaction masks in {0,1,2}
 * replace the visited point set, cost O(n^3 3^n)).
 *
 * Conventions shared by every entry point
 *   - Result c(V) is the bare combinatorial sum: sum over connected decorated
 *     covers of the 2n points (point i and i+n belong to vertex i) of
 *     prod_loops ( -sum_l prod G0^l(edge) prod_{shifts on the loop} (-sigma_l) ),
 *     with at most one shift point per vertex (counter-term, Methods A shifted
 *     action) whose weight takes the flavor of its partner's loop (Alg. 3).
 *     Prefactors (-U)^n / n! are the caller's business.
 *   - A "symmetric" run (all flavors share one propagator and one shift)
 *     carries one matrix per configuration and weight N_f per closed loop
 *     (Alg. 2 multiplies every close by N_f).
 *   - Device pointers (d_*) are caller-owned CUDA device memory; host
 *     pointers (h_*) are read before the call returns.  Every call is
 *     asynchronous on `stream` (a cudaStream_t, 0 = legacy default stream).
 *     Argument errors are returned synchronously; errors detected on the
 *     device (order out of range, non-finite result) are recorded in a
 *     per-stream status word reported by cos_sync_status().
 *   - No entry point falls back to host arithmetic: without a usable CUDA
 *     device the calls return COS_ERR_CUDA.
 *   - Calls enqueued on different streams of one device use different
 *     internal workspaces and may overlap; calls on one stream serialize.
 */
#ifndef COS_H
#define COS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define COS_NMAX 12      /* largest order n supported (3^12 interaction masks) */
#define COS_MAX_FLAVORS 8

typedef void *cos_stream_t; /* cudaStream_t */

typedef enum {
    COS_OK = 0,
    COS_ERR_ARG = -1,           /* null pointer, negative count, bad enum */
    COS_ERR_ORDER = -2,         /* an order n < 1 or n > n_max (or > COS_NMAX) */
    COS_ERR_CUDA = -3,          /* a CUDA call failed (message: cos_last_error) */
    COS_ERR_TIMEOUT = -4,       /* reserved: no call of this library waits on the device (the
                                   persistent kernels take batches from an atomic counter and
                                   never spin on a flag), so none returns it */
    COS_ERR_NONFINITE = -5,     /* a result was NaN or infinite */
    COS_ERR_UNIMPLEMENTED = -6,
    COS_ERR_NOMEM = -7          /* device workspace could not be allocated */
} cos_status;

typedef enum {
    COS_FP64 = 0,   /* every step in FP64 */
    COS_MIXED = 1,  /* clow extension in FP32 with FP32 accumulation; loop-closing
                       sums as compensated FP32 sums (Dot2 on close matrices split into
                       FP32 pairs, about 47 bits) widened and added in FP64 once per mask
                       (the bipartite sweep at n_max = 9: FP64 sums on exactly widened
                       states); seeds of new loops and the sink formed in FP64 */
    COS_DF64 = 2    /* double-float: states, matrices, extension and loop-closing sums as
                       unevaluated pairs hi + lo of FP32 numbers (about 48 bits), each dot
                       product a compensated (TwoSum / FMA TwoProduct) accumulation on the
                       FP32 pipe; only the output is formed in FP64.  The paper answers
                       cancellation with software extended precision (double-double, at 3-5x
                       the cost: Methods, fast generation of 3^n minors; Discussion); this is
                       that remedy mapped onto B300's FP32 units, which retire 64 lane
                       operations for each FP64 one.  Forward entry points only (the
                       gradient is FP64). */
} cos_precision;

/* Square-lattice model (Methods A): dispersion
 *   xi_l(k) = -2t [cos k_x + cos k_y] - mu_l + alpha_l,  k = 2 pi m / L,
 * shift weight sigma_l = alpha_l / U (equal-time shift of SB-CoS, Methods A).
 * mu and alpha are host arrays of n_flavors values.  The imaginary-time grid
 * holds n_tau points tau_m = m beta / (n_tau - 1), m = 0 .. n_tau - 1. */
typedef struct {
    int L;
    double t, beta, U;
    int n_flavors;
    const double *mu;
    const double *alpha;
    int n_tau;
} cos_model;

/* Honeycomb-lattice model (Methods A, bipartite lattices): L x L unit cells of two sites
 * (sublattices A, B), Bloch Hamiltonian per flavor l
 *   H_l(k) = [[delta_l - (mu_l - alpha_l), eps(k)], [conj(eps(k)), -delta_l - (mu_l - alpha_l)]],
 *   eps(k) = -t (1 + exp(i k.b1) + exp(i k.b2)),  k.b1 = 2 pi m_1 / L, k.b2 = 2 pi m_2 / L.
 * Shift weights per (flavor, sublattice): sigma_{l,A} = (alpha_l + delta_l) / U,
 * sigma_{l,B} = (alpha_l - delta_l) / U (the sublattice-dependent equal-time shift).
 * mu, alpha and delta are host arrays of n_flavors values; the tau grid is the square
 * lattice's. */
typedef struct {
    int L;
    double t, beta, U;
    int n_flavors;
    const double *mu;
    const double *alpha;
    const double *delta;
    int n_tau;
} cos_honeycomb_model;

#define COS_BIP_NMAX 9    /* largest order of the bipartite DP (4^n interaction masks) */

typedef struct cos_tables cos_tables; /* opaque; owns device propagator tables */

typedef struct {
    int L, n_tau, n_flavors;
    int symmetric;          /* 1: one table and weight n_flavors per loop */
    int n_mat;              /* matrices per configuration: 1 if symmetric else n_flavors */
    double beta, U;
    double sigma[COS_MAX_FLAVORS];
    const double *d_G;      /* [n_mat][L*L][n_tau]  G0(r, tau_m), r = x + L y */
    const double *d_dGdmu;  /* same layout, d G0 / d mu; NULL until a gradient call */
    int bipartite;          /* 1: honeycomb tables, d_G = [n_mat][2][2][L*L][n_tau] (s, t, R, tau) */
    double sigma2[COS_MAX_FLAVORS][2];   /* bipartite: shift weight per (flavor, sublattice) */
} cos_tables_info;

/* ------------------------------------------------------------------ K-TAB
 * Tabulates, on the device, for every distinct flavor l
 *   G0_l(r, tau_m) = -(1/L^2) sum_k cos(k.r) exp(-xi tau_m)(1 - n_F(xi))
 * (Methods A dispersion; G0 = -<T c c^+>, antiperiodic in tau), stored at
 * tau_m for m = 0 .. n_tau-1 (G(0^+) first, G(beta^-) last).
 * model      host struct; copied.  L in [1, 256], n_tau in [2, 65536],
 *            n_flavors in [1, COS_MAX_FLAVORS], beta > 0, U != 0.
 * out        receives a new table object owned by the caller (cos_free_tables).
 * The call returns after the tables are complete (it synchronizes `stream`). */
cos_status cos_build_propagators(const cos_model *model, cos_stream_t stream, cos_tables **out);
cos_status cos_free_tables(cos_tables *tables);
cos_status cos_get_tables_info(const cos_tables *tables, cos_tables_info *info);
/* Copies a whole table ([n_mat][L*L][n_tau] doubles; honeycomb: [n_mat][2][2][L*L][n_tau])
 * into caller device memory d_dst, asynchronously on `stream`.  which = 0: G0; which = 1:
 * dG0/dmu (built on first request; square tables only). */
cos_status cos_copy_table(const cos_tables *tables, int which, double *d_dst, cos_stream_t stream);

/* ------------------------------------------------------------------ K-GATHER
 * M^l[i][j] = G0_l(r_i - r_j, tau_i - tau_j) for every configuration (Methods A:
 * the matrix entries g(X_i, X_j) of the diagrammatic expansion), by linear
 * interpolation in tau; a difference dt <= 0 (equal times and the diagonal
 * included) is read as -G0(r, dt + beta), i.e. equal times at tau = 0^-.
 * d_order[c]  n_c in [1, COS_NMAX]
 * d_offset[c] index of the first vertex of configuration c in d_site / d_tau
 * d_site[k]   x + L*y in [0, L^2);  d_tau[k] in [0, beta)
 * d_moff[c]   offset (in doubles) of configuration c's block [n_mat][n_c][n_c]
 *             in d_M (row-major, row i = first vertex).
 * Out-of-range orders or sites set the device status (COS_ERR_ORDER / COS_ERR_ARG). */
cos_status cos_gather(const cos_tables *tables, int n_cfg, const int32_t *d_order,
                      const int64_t *d_offset, const int32_t *d_site, const double *d_tau,
                      const int64_t *d_moff, double *d_M, cos_stream_t stream);

/* ------------------------------------------------------------------ K-DP
 * Connected sum of every configuration from explicit matrices (the DP
 * proper: seed, clow extension, loop closing, sink).
 * n_cfg        number of configurations (0 allowed)
 * n_max        largest order present (sizes the workspace); orders must lie
 *              in [1, n_max], n_max <= COS_NMAX
 * d_order[c]   order n_c
 * d_moff[c]    offset of configuration c's matrices [n_mat][n_c][n_c] in d_M
 * n_mat        matrices per configuration: 1 (symmetric) or the number of
 *              flavors (broken), <= COS_MAX_FLAVORS
 * loop_weight  weight of a closed loop beyond the flavor sum: N_f for a
 *              symmetric run (n_mat = 1), 1 for a broken run
 * h_sigma      host array of n_mat shift weights sigma_l, or NULL (no shifts)
 * d_out[c]     connected sum c(V) of configuration c
 * d_abs_mass   NULL, or d_abs_mass[c] = the same DP on |M|, |sigma| with every
 *              sign +, an upper bound of sum |term| (for error statements)
 * Configurations of different orders share one persistent launch (largest
 * order first, one CTA per batch of configurations). */
cos_status cos_connected_sum_matrices(int n_cfg, int n_max, const int32_t *d_order,
                                      const int64_t *d_moff, int n_mat, int loop_weight,
                                      const double *h_sigma, const double *d_M,
                                      cos_precision precision, double *d_out,
                                      double *d_abs_mass, cos_stream_t stream);

/* Same computation as cos_connected_sum_matrices for callers that cannot allocate device
 * memory (no counterpart in the paper: it exists for integrations such as a plug-in that
 * receives a stream and buffers but no allocator, or a process whose device memory is owned
 * by a pool).  It calls no cudaMalloc / cudaFree and no allocating library routine: all
 * scratch (planner tables, work queue, DP structure, layer ring) lives in one fixed device
 * array of 128 MiB that every GPU loading the library holds until the process exits.
 *   - Limits: n_max <= 10, and the batch must fit the array (roughly 20 B per configuration
 *     plus one layer ring of 2 x max-layer-slots x 32 x 8 B); larger requests return
 *     COS_ERR_ORDER / COS_ERR_ARG with a message, without launching anything.
 *   - The array is device memory of this library's module, loaded on a device by the first
 *     call there (under the runtime's default lazy module loading): that call takes the
 *     128 MiB from the device's free memory, then sets the array up (device address, DP
 *     structure copy, synchronizing `stream` once).  Make that first call before a memory
 *     pool claims the device's free memory, and before any stream capture; later calls
 *     allocate nothing.
 *   - Mixed and double-float run the one-configuration-per-lane forward kernels (the regular
 *     call runs the pair kernels), in launch shapes tuned for the regular call.
 *   - Every call reuses the same array and leaves its contents behind; calls whose work
 *     overlaps on the GPU (other streams, other host threads) race with each other.
 *   - Outputs are set to NaN first; a configuration whose order lies outside [1, n_max]
 *     keeps NaN.  There is no device status word on this path. */
cos_status cos_connected_sum_matrices_noalloc(int n_cfg, int n_max, const int32_t *d_order,
                                              const int64_t *d_moff, int n_mat, int loop_weight,
                                              const double *h_sigma, const double *d_M,
                                              cos_precision precision, double *d_out,
                                              double *d_abs_mass, cos_stream_t stream);

/* Gather + DP from vertex coordinates (arguments as in cos_gather and
 * cos_connected_sum_matrices; sigma and the loop weight come from the tables). */
cos_status cos_connected_sum_batch(const cos_tables *tables, int n_cfg, int n_max,
                                   const int32_t *d_order, const int64_t *d_offset,
                                   const int32_t *d_site, const double *d_tau,
                                   cos_precision precision, double *d_out,
                                   double *d_abs_mass, cos_stream_t stream);

/* ------------------------------------------------------------------ bipartite lattices
 * Connected sums summed over every sublattice assignment of the vertices (Methods A,
 * bipartite lattices, strategy (i)) by the sublattice-resolved merged DP (Results A; Alg. 1-2):
 * the interaction mask keeps the sublattice of each half-visited vertex, so the 2^n
 * assignments share one sweep.
 *
 * Two-band tables for the honeycomb model: for every distinct flavor l the real 2 x 2 matrix
 *   G_l(R, tau_m) = -(1/L^2) sum_k exp(i k.R) exp(-H_l(k) tau_m)(1 - n_F(H_l(k))),
 * R = r_1 + L r_2 in unit-cell coordinates, tau_m as in cos_build_propagators.  Same
 * ownership and synchronization as cos_build_propagators; the tables serve the bipartite
 * entry points only. */
cos_status cos_build_propagators_honeycomb(const cos_honeycomb_model *model, cos_stream_t stream,
                                           cos_tables **out);

/* M4^l[(i,s)][(j,t)] = G_l^{st}(R_i - R_j, tau_i - tau_j) (same interpolation and dt <= 0 reading
 * as cos_gather).  Per configuration c the block [n_mat][2 n_c][2 n_c] (row index i*2 + s,
 * column j*2 + t, s, t = 0 for A, 1 for B) starts at d_moff[c] in d_M4.  d_site[k] is the unit
 * cell r_1 + L r_2 in [0, L^2).  Orders in [1, COS_BIP_NMAX]; a configuration with another
 * order or a negative d_moff[c] is skipped and reported through the status word. */
cos_status cos_gather_bipartite(const cos_tables *tables, int n_cfg, const int32_t *d_order,
                                const int64_t *d_offset, const int32_t *d_site, const double *d_tau,
                                const int64_t *d_moff, double *d_M4, cos_stream_t stream);

/* ------------------------------------------------------------------ one call per operation
 * Every connected sum this library computes is described by a cos_problem: the lattice, the
 * weight of a diagram, the precision, and the input -- vertex coordinates with tables, or
 * explicit matrices.  cos_forward, cos_grad and cos_subsets take it.  cos_connected_sum_matrices,
 * cos_connected_sum_batch and cos_connected_sum_grad are the square-lattice, loop-weight
 * cases of cos_forward / cos_grad under their own names.
 *
 * lattice
 *   COS_SQUARE     one site per vertex; matrices [n_mat][n_c][n_c] per configuration (the
 *                  layout of cos_gather).
 *   COS_BIPARTITE  the connected sum summed over every sublattice assignment of the vertices
 *                  (Methods A, bipartite lattices, strategy (i)) by the sublattice-resolved
 *                  merged DP (Results A; Alg. 1-2): the interaction mask keeps the sublattice of
 *                  each half-visited vertex, so the 2^n assignments share one sweep.  Matrices
 *                  [n_mat][2 n_c][2 n_c] per configuration (the layout of cos_gather_bipartite);
 *                  orders up to COS_BIP_NMAX.
 * weights
 *   COS_LOOPS         CoS: -1 and a flavor weight per closed loop (Alg. 2-3 merged, Results A):
 *                     the flavor sum over the n_mat matrices times loop_weight (N_f for one
 *                     symmetric matrix).  Shift weights h_shift: square NULL or [n_mat] sigma_l;
 *                     bipartite NULL or [n_mat][2] sigma_{l,s} (flavor, sublattice).
 *   COS_DETERMINANTS  SU(2) with determinant weights (the interaction (n_up - alpha_up)
 *                     (n_dn - alpha_dn), Methods A): the sum of all diagrams of a vertex set S is
 *                     a(S) = det(A_up[S]) det(A_dn[S]) (summed over sublattice assignments on a
 *                     bipartite lattice), A_b = M_b - diag(alpha_b), and the output is its
 *                     connected part c(V) (the subset subtraction of Methods A), computed by the
 *                     DP without cycle factors of Results A and Alg. 1 (interaction masks only,
 *                     nonphysical clow sequences kept, they cancel).  Two matrices per
 *                     configuration, spin up then spin down (n_mat and loop_weight are not read);
 *                     h_shift: square NULL or [2] alpha_b, bipartite NULL or [2][2] alpha_{b,s}.
 *                     For alpha = 0 the COS_LOOPS sum of the same matrices with n_mat = 2 and
 *                     loop_weight = 1 is 2^n c(V).
 * input
 *   tables != NULL  vertex coordinates d_offset, d_site, d_tau (as cos_gather); the matrices are
 *                   gathered into the library's workspace.  Loop weights take n_mat, the loop
 *                   weight and the shift weights from the tables (h_shift must be NULL);
 *                   determinant weights need two-flavor tables built with alpha = 0 (tables
 *                   collapsed to one matrix for equal chemical potentials serve both spins) and
 *                   take their diagonal shifts from h_shift.  Square-lattice tables of
 *                   cos_build_propagators for COS_SQUARE, honeycomb tables for COS_BIPARTITE.
 *   tables == NULL  explicit matrices d_M at d_moff[c] (in doubles), n_mat and loop_weight as
 *                   above.
 * precision: COS_FP64, COS_MIXED (FP32 extension, compensated loop closes) or COS_DF64 for
 *   cos_forward; COS_FP64 for cos_grad and cos_subsets (COS_ERR_UNIMPLEMENTED otherwise).
 * Orders must lie in [1, n_max], n_max <= COS_NMAX (COS_BIP_NMAX on the bipartite lattice).
 * Errors: invalid descriptors return COS_ERR_ARG / COS_ERR_ORDER synchronously; device-detected
 * errors land in the stream's status word (cos_sync_status). */
typedef enum { COS_SQUARE = 0, COS_BIPARTITE = 1 } cos_lattice;
typedef enum { COS_LOOPS = 0, COS_DETERMINANTS = 1 } cos_weights;

typedef struct {
    cos_lattice lattice;
    cos_weights weights;
    cos_precision precision;
    int n_cfg;                  /* configurations (0 allowed) */
    int n_max;                  /* largest order present */
    const int32_t *d_order;     /* [n_cfg] orders n_c */
    const cos_tables *tables;   /* coordinates form: the tables, else NULL */
    const int64_t *d_offset;    /* coordinates form: first vertex of each configuration */
    const int32_t *d_site;      /* coordinates form: site (unit cell) of every vertex */
    const double *d_tau;        /* coordinates form: imaginary time of every vertex */
    const int64_t *d_moff;      /* matrices form: offset of each configuration's matrices */
    const double *d_M;          /* matrices form: the matrices */
    int n_mat;                  /* matrices form, COS_LOOPS: matrices per configuration */
    int loop_weight;            /* matrices form, COS_LOOPS: weight of a loop beyond the flavor sum */
    const double *h_shift;      /* host shift weights (see weights), NULL = none */
} cos_problem;

/* Connected sums: d_out[c] = c(V) of configuration c; d_abs_mass NULL, or the same DP on |M|
 * and |shifts| with every sign + (an upper bound of the sum of |terms|, for error
 * statements).  Configurations of different orders share one persistent launch. */
cos_status cos_forward(const cos_problem *p, double *d_out, double *d_abs_mass, cos_stream_t stream);

/* Gradients by the reverse (adjoint) DP -- the adjoint of Alg. 2-3 (loop weights) or Alg. 1
 * (determinant weights) as merged in Results A; the paper computes no gradients:
 *   d_gout[c]  dLoss/dc of configuration c (the vector the gradient is contracted with);
 *   d_out      NULL or receives c;
 *   d_gM       NULL or dLoss/dM: matrices form at d_moff (d_gmoff must be NULL); coordinates
 *              form at d_gmoff[c] ([n_mat][n_c][n_c], bipartite [n_mat][2 n_c][2 n_c];
 *              determinant weights both spin blocks, also for collapsed tables);
 *   d_gshift   NULL or dLoss/d(h_shift) per configuration: [n_cfg][n_mat] sigma (square
 *              loops), [n_cfg][n_mat][2] sigma2 (bipartite loops), [n_cfg][2] alpha
 *              (= -trace of dLoss/dM_b) and [n_cfg][2][2] alpha2 (= minus the sublattice
 *              traces) for determinant weights; computed also at zero shifts.  Coordinates
 *              form of loop weights: must be NULL (their shifts come from the tables, see
 *              d_galpha);
 *   d_gmu      coordinates form: NULL or [n_cfg][n_flavors] dLoss/dmu_l = sum_ij dLoss/dM^l_ij
 *              dM^l_ij/dmu_l (the gather's interpolation of a dG/dmu table, built on first
 *              use, synchronizing the stream); for collapsed tables the common derivative is
 *              split evenly over the flavors;
 *   d_galpha   coordinates form of loop weights: NULL or [n_cfg][n_flavors] dLoss/dalpha_l =
 *              -(that sum) + dLoss/dsigma_l / U (sigma_l = alpha_l / U; on the honeycomb
 *              lattice the two sublattice shifts (alpha_l +- delta_l) / U); must be NULL for
 *              determinant weights (their alpha is h_shift).
 * The forward sweep is re-run with every layer kept and walked backwards (see the checkpoint
 * plans below for the memory it takes); FP64. */
cos_status cos_grad(const cos_problem *p, const double *d_gout, double *d_out, double *d_gM,
                    const int64_t *d_gmoff, double *d_gshift, double *d_gmu, double *d_galpha,
                    cos_stream_t stream);

/* Connected sums of every vertex subset (Methods A: the subset recursion between the sum over
 * all decorated covers a(S) and the sum over connected ones c(S)).  One configuration of n
 * vertices then yields every lower order, as a CDet evaluation does.  Matrices form only.
 *   d_c  [n_cfg][2^n_max]  c(S) at index c * 2^n_max + S, bit i of S = vertex i.
 *        c(empty) = 0, and sets holding a vertex >= the configuration's order are 0.
 *        all_roots = 1: every nonempty S.  The merged DP rooted at vertex m on the trailing
 *          principal submatrices M^l[m.., m..] gives c(S) for every S whose smallest vertex is m
 *          (from the closes of the masks with no half-visited vertex; on a bipartite lattice
 *          summed over the sublattice assignments of S, with determinant weights the connected
 *          part of det(A_up[S]) det(A_dn[S])); all roots of all configurations run as one batch
 *          of derived problems, about 1.5 times the work of the order-n DP at n = 10.
 *        all_roots = 0: only the sets containing vertex 0, a by-product of the order-n DP
 *          (which then also closes the masks it otherwise drops); the other entries are NaN.
 *   d_a  NULL, or [n_cfg][2^n_max] receiving a(S) = sum_{T subset of S, min S in T}
 *        c(T) a(S \ T), a(empty) = 1 (with determinant weights det(A_up[S]) det(A_dn[S])),
 *        evaluated in FP64 on the GPU; needs all_roots = 1.
 * Precision applies to the DP (square loop weights: any; otherwise COS_FP64); the recursion
 * for a is FP64.  Workspace: besides the DP's, all_roots = 1 holds n_cfg * n_max derived
 * problems and their submatrices.  A device-detected order error is reported as for the
 * other entry points; the outputs of that call are then undefined. */
cos_status cos_subsets(const cos_problem *p, int all_roots, double *d_c, double *d_a, cos_stream_t stream);

/* ------------------------------------------------------------------ adjoint DP
 * cos_connected_sum_grad (the gradient of cos_connected_sum_batch) is cos_grad with a
 * square-lattice, loop-weight cos_problem in the coordinates form; the descriptor call also
 * takes explicit matrices, bipartite lattices and determinant weights. */

/* Memory of the gradient calls.  The reverse sweep needs the forward state of every layer;
 * each adjoint overwrites the forward state it was formed from, so the kept layers are the
 * whole workspace: about (states per flavor array) x 32 lanes x 8 B per CTA, 181 MB at n = 10
 * and 2.2 GB at n = 12 on the square lattice, 3.3 GB at n = 9 on the bipartite one (with
 * 2 x 4 n^2 x 32 doubles of gradient accumulators per CTA there at n = 9).  Where free device
 * memory cannot hold that for every CTA, layers are
 * checkpointed (the reverse of Alg. 2-3 with the forward recomputed per segment): a set of
 * checkpoint layers is kept, and the layers between two checkpoints are re-run from the first
 * before they are reversed.  The launcher picks, per order, the grid and checkpoint set that
 * give the most throughput within 85 % of the free memory.  The environment variable
 * COS_GRAD_CHECKPOINT=1 forces the least-storage plan at every order, =0 keeps every layer.
 *
 * cos_grad_checkpoint_plan (host only, no device): the square lattice's plan of order n for a budget of
 * slots_budget state slots per lane (0: the least storage): *ck_mask bit l = layer l is a
 * checkpoint (layers are numbered by visited points, 1 .. 2n; 0 = every layer kept),
 * *store_slots = slots per lane kept (checkpoints plus the largest segment between two),
 * *recompute_fma = multiply-adds of one flavor array re-run.  COS_ERR_ARG if nothing fits. */
cos_status cos_grad_checkpoint_plan(int n, int64_t slots_budget, uint32_t *ck_mask, int64_t *store_slots,
                                    int64_t *recompute_fma);

/* Gradient from vertex coordinates, with the chain rule through the tables:
 *   dc/dmu_l    = sum_ij dc/dM^l_ij  dM^l_ij/dmu_l  (same interpolation of the dG0/dmu table
 *                 as the gather), the tables' xi depends on mu_l - alpha_l;
 *   dc/dalpha_l = -(that sum) + dc/dsigma_l / U   (sigma_l = alpha_l / U, Methods A).
 * For symmetric tables the common derivative is split evenly over the n_flavors flavors.
 * d_gM / d_gmoff: NULL, or dLoss/dM written at d_gmoff[c] as [n_mat][n_c][n_c].
 * d_gmu, d_galpha: NULL or [n_cfg][n_flavors] (per configuration, scaled by d_gout[c]).
 * Builds the dG0/dmu table on first use. */
cos_status cos_connected_sum_grad(const cos_tables *tables, int n_cfg, int n_max, const int32_t *d_order,
                                  const int64_t *d_offset, const int32_t *d_site, const double *d_tau,
                                  const double *d_gout, double *d_out, double *d_gM,
                                  const int64_t *d_gmoff, double *d_gmu, double *d_galpha,
                                  cos_stream_t stream);

/* ------------------------------------------------------------------ graphs and tuning
 * A plan freezes one batch (fixed device addresses of inputs and outputs) into a CUDA graph:
 * device planner, gather (batch plan), persistent DP kernel(s).  Creation runs the call once
 * eagerly on `stream` (results valid afterwards), then captures it; the plan owns a private
 * workspace, so plans never share scratch with each other or with direct calls.
 * cos_plan_launch replays it with one cudaGraphLaunch on any stream; cos_plan_status
 * synchronizes that stream and reports (and clears) the plan's device status word. */
typedef struct cos_plan cos_plan;
cos_status cos_plan_create_batch(const cos_tables *tables, int n_cfg, int n_max, const int32_t *d_order,
                                 const int64_t *d_offset, const int32_t *d_site, const double *d_tau,
                                 cos_precision precision, double *d_out, double *d_abs_mass,
                                 cos_stream_t stream, cos_plan **out);
cos_status cos_plan_create_matrices(int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                                    int n_mat, int loop_weight, const double *h_sigma, const double *d_M,
                                    cos_precision precision, double *d_out, double *d_abs_mass,
                                    cos_stream_t stream, cos_plan **out);
cos_status cos_plan_launch(cos_plan *plan, cos_stream_t stream);
cos_status cos_plan_status(cos_plan *plan, cos_stream_t stream);
cos_status cos_plan_grid(const cos_plan *plan, int *grid);   /* persistent CTAs of the plan */
cos_status cos_plan_destroy(cos_plan *plan);

/* Launch shape of the DP kernel per (order n_max of the launch, precision, matrices per
 * configuration): warps per CTA (1..16; 1..20 for mixed and double-float), resident CTAs per SM
 * (1..8) and whether a warp
 * prefetches the states of its next mask while it computes the current one (prefetch:
 * 0 = off, 1 = into L2, 2 = into L1; 3 = the mixed and double-float kernels pull each next row's
 * states into L1 while a row computes, 4 = 3 plus the next mask into L2; the FP64 kernel treats
 * 3 and 4 as 2).  A launch mixing
 * orders uses the shape of its largest order, which dominates its work (a factor 3-4 per
 * order).  cos_autotune times every shape the occupancy calculator admits on n_cfg
 * synthetic configurations of order n (device buffers allocated for the run), installs the
 * fastest, and appends "n precision n_mat warps ctas ms prefetch" to the file named by the
 * environment variable COS_TUNE_OUT, if set.  At the first launch a process reads the
 * tuning file named by COS_TUNE_FILE (the Python binding points it at the package's
 * tuning_b300.txt unless the caller set it). */
cos_status cos_set_tuning(int n, cos_precision precision, int n_mat, int warps, int ctas_per_sm, int prefetch);
cos_status cos_get_tuning(int n, cos_precision precision, int n_mat, int *warps, int *ctas_per_sm,
                          int *prefetch /* nullable */);
cos_status cos_autotune(int n, int n_mat, int loop_weight, int shifts, cos_precision precision, int n_cfg,
                        cos_stream_t stream, int *best_warps, int *best_ctas, int *best_prefetch,
                        double *best_ms);

/* ------------------------------------------------------------------ status
 * Synchronizes `stream`, returns and clears the device status word of the
 * calls enqueued on it (COS_OK if none failed). */
cos_status cos_sync_status(cos_stream_t stream);

/* Frees the device workspace the library keeps for `stream` on the current device (layer
 * rings and kept layers, gathered matrices, planner tables; it grows to the largest call made
 * on the stream and stays allocated between calls).  Synchronizes the stream and reports its
 * status word first, as cos_sync_status; the next call on the stream allocates afresh.  Plans
 * and the no-allocation entry point keep their own workspaces and are not affected. */
cos_status cos_release_workspace(cos_stream_t stream);
const char *cos_status_string(cos_status status);
/* Message of the last synchronous error in this thread ("" if none). */
const char *cos_last_error(void);

/* ------------------------------------------------------------------ structure (host only)
 * Counts of the merged DP for order n (no device needed): interaction masks
 * (mu_0 >= 1), state slots (head x endpoint per mask), reachable states, and
 * the FP64 multiply-adds of one flavor array (extension dot products and
 * loop-closing sums over reachable states). */
typedef struct {
    int n;
    int64_t masks;
    int64_t slots;
    int64_t max_layer_slots;
    int64_t states;
    int64_t fma_ext;        /* clow extension multiply-adds */
    int64_t fma_close;      /* loop-closing multiply-adds */
    int64_t mul_shift;      /* shift transitions (one per row and untouched vertex); they ride on
                               the shifted diagonal of the extension matrices, no extra work */
} cos_structure_info;

cos_status cos_structure(int n, cos_structure_info *info);

/* Counts of the bipartite structure at order n (host only): masks, slots (4 |H| |A| per
 * mask), max_layer_slots, reachable states and multiply-adds per flavor array. */
cos_status cos_bipartite_structure(int n, cos_structure_info *info);

#ifdef __cplusplus
}
#endif
#endif /* COS_H */
