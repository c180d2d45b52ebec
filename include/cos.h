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
                       sums, seeds of new loops and the sink in FP64 */
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

/* ------------------------------------------------------------------ all subsets
 * Connected sums of every vertex subset (Methods A: the subset recursion between the sum over
 * all decorated covers a(S) and the sum over connected ones c(S)).  One configuration of n
 * vertices then yields every lower order, as a CDet evaluation does.
 *   d_c  [n_cfg][2^n_max]  c(S) at index c * 2^n_max + S, bit i of S = vertex i.
 *        c(empty) = 0, and sets holding a vertex >= the configuration's order are 0.
 *        all_roots = 1: every nonempty S.  The merged DP of Results A rooted at vertex m on the
 *          trailing principal submatrices M^l[m.., m..] gives c(S) for every S whose smallest
 *          vertex is m (from the closes of the masks with no half-visited vertex); all roots of
 *          all configurations run as one batch of derived problems, about 1.5 times the work
 *          of the order-n DP at n = 10.
 *        all_roots = 0: only the sets containing vertex 0, a by-product of the order-n DP
 *          (which then also closes the masks it otherwise drops); the other entries are NaN.
 *   d_a  NULL, or [n_cfg][2^n_max] receiving a(S) = sum_{T subset of S, min S in T}
 *        c(T) a(S \ T), a(empty) = 1, evaluated in FP64 on the GPU; needs all_roots = 1.
 * Other arguments as cos_connected_sum_matrices (precision applies to the DP; the recursion
 * for a is FP64).  Workspace: besides the DP's, all_roots = 1 holds n_cfg * n_max derived
 * problems and their submatrices (n_mat * n_max (n_max + 1) (2 n_max + 1) / 6 doubles per
 * configuration).  A device-detected order error is reported as for the other entry points;
 * the outputs of that call are then undefined. */
cos_status cos_connected_sum_subsets(int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                                     int n_mat, int loop_weight, const double *h_sigma, const double *d_M,
                                     cos_precision precision, int all_roots, double *d_c, double *d_a,
                                     cos_stream_t stream);

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

/* Bipartite connected sums of explicit matrices: d_M4 as written by cos_gather_bipartite
 * (blocks [n_mat][2 n_c][2 n_c] at d_moff[c]); h_sigma2 = NULL or host [n_mat][2] shift weights
 * per (flavor, sublattice).  n_max <= COS_BIP_NMAX; precision COS_FP64, COS_MIXED (FP32
 * extension, FP64 close, as on the square lattice) or COS_DF64.  Other arguments, outputs and errors as
 * cos_connected_sum_matrices (d_abs_mass: the same DP on |M4|, |sigma| with all signs +). */
cos_status cos_connected_sum_bipartite_matrices(int n_cfg, int n_max, const int32_t *d_order,
                                                const int64_t *d_moff, int n_mat, int loop_weight,
                                                const double *h_sigma2, const double *d_M4,
                                                cos_precision precision, double *d_out,
                                                double *d_abs_mass, cos_stream_t stream);

/* Gradient of the bipartite sums by the reverse sweep (the forward sweep re-run with every
 * layer kept, then walked backwards): d_gout[c] = dLoss/dc; d_out NULL or receives c;
 * d_gM4 NULL or dLoss/dM4 (layout and offsets of d_M4); d_gsigma2 NULL or [n_cfg][n_mat][2]
 * dLoss/dsigma_{l,s} (also at sigma = 0).  n_max <= COS_BIP_NMAX (up to 8 the dLoss/dM4
 * accumulators sit in shared memory beside the two matrix copies, at 9 in the workspace:
 * 4 (2 n_max)^2 x 32 doubles per CTA more); FP64.  Other arguments as
 * cos_connected_sum_bipartite_matrices. */
cos_status cos_connected_sum_bipartite_matrices_grad(int n_cfg, int n_max, const int32_t *d_order,
                                                     const int64_t *d_moff, int n_mat, int loop_weight,
                                                     const double *h_sigma2, const double *d_M4, const double *d_gout,
                                                     double *d_out, double *d_gM4, double *d_gsigma2,
                                                     cos_stream_t stream);

/* Gather + bipartite DP from vertex coordinates (honeycomb tables; the loop weight is
 * n_flavors for symmetric tables, else 1). */
cos_status cos_connected_sum_bipartite_batch(const cos_tables *tables, int n_cfg, int n_max,
                                             const int32_t *d_order, const int64_t *d_offset,
                                             const int32_t *d_site, const double *d_tau,
                                             cos_precision precision, double *d_out,
                                             double *d_abs_mass, cos_stream_t stream);

/* Every vertex subset on a bipartite lattice (the all-subsets mode of
 * cos_connected_sum_subsets on the sublattice-resolved sweep): d_c[c * 2^n_max + S] = c(S),
 * the connected sum of the sub-configuration S summed over its sublattice assignments (the
 * close of a mask with every vertex of S fully visited and no half-visited vertex, Methods A
 * and Alg. 1-2), and with d_a, a(S) by the subset exponential.  Layout of d_M4 / h_sigma2 as
 * cos_connected_sum_bipartite_matrices; all_roots, layout of d_c / d_a, workspace and errors
 * as cos_connected_sum_subsets; n_max <= COS_BIP_NMAX; COS_FP64 only (COS_ERR_UNIMPLEMENTED
 * for the other precisions). */
cos_status cos_connected_sum_bipartite_subsets(int n_cfg, int n_max, const int32_t *d_order,
                                               const int64_t *d_moff, int n_mat, int loop_weight,
                                               const double *h_sigma2, const double *d_M4,
                                               cos_precision precision, int all_roots, double *d_c,
                                               double *d_a, cos_stream_t stream);

/* ------------------------------------------------------------------ SU(2) determinant weights
 * Connected sums of an SU(2) model whose diagrams are weighted by determinants (the
 * interaction (n_up - alpha_up)(n_dn - alpha_dn), Methods A): the sum of all diagrams of a
 * vertex set S is a(S) = det(A_up[S]) det(A_dn[S]) (summed over sublattice assignments on a
 * bipartite lattice), A_b = M_b - diag(alpha_b), and the output is its connected part c(V)
 * (the subset subtraction of Methods A).  Computed by the DP without cycle factors of Results
 * A and Alg. 1: only the interaction mask is tracked, nonphysical clow sequences are kept and
 * cancel, and every vertex has a spin-up point (block 0) and a spin-down point (block 1).
 * For alpha = 0 the CoS sum of the same matrices with n_mat = 2, loop_weight = 1 is 2^n c(V).
 *
 * Square lattice: d_M holds per configuration the two blocks [2][n_c][n_c] (spin up, spin
 * down) at d_moff[c], as written by cos_gather for two-flavor tables; h_alpha = NULL or
 * host [2] diagonal shifts.  Precision COS_FP64, COS_MIXED (FP32 extension, FP64 close) or
 * COS_DF64.  d_abs_mass: NULL, or the same DP on |M| with |alpha| added to the diagonal and
 * every sign + (an upper bound on the sum of |terms| of the DP, nonphysical clows included).
 * Other arguments and errors as cos_connected_sum_matrices. */
cos_status cos_connected_det_matrices(int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                                      const double *h_alpha, const double *d_M, cos_precision precision,
                                      double *d_out, double *d_abs_mass, cos_stream_t stream);

/* Gather + determinant-weight sweep from vertex coordinates: SU(2) tables of
 * cos_build_propagators (two flavors: spin up, spin down; tables collapsed to one matrix for
 * equal chemical potentials serve both blocks), built with alpha = 0 (the diagonal shifts of
 * determinant weights are h_alpha, not the tables' dispersion shift).  Other arguments as
 * cos_connected_sum_batch and cos_connected_det_matrices; COS_ERR_ARG for tables with another
 * flavor count. */
cos_status cos_connected_det_batch(const cos_tables *tables, int n_cfg, int n_max, const int32_t *d_order,
                                   const int64_t *d_offset, const int32_t *d_site, const double *d_tau,
                                   const double *h_alpha, cos_precision precision, double *d_out,
                                   double *d_abs_mass, cos_stream_t stream);

/* Gradient of the square-lattice determinant-weight sums by the reverse sweep (the adjoint of
 * Alg. 1 as merged above; the forward sweep is re-run with every layer kept):
 * d_gout[c]  dLoss/dc;  d_out NULL or receives c;  d_gM NULL or dLoss/dM at d_moff[c] as
 * [2][n_c][n_c];  d_galpha NULL or [n_cfg][2] dLoss/dalpha_b (= -trace of dLoss/dM_b).
 * Other arguments as cos_connected_det_matrices; FP64 only. */
cos_status cos_connected_det_matrices_grad(int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                                           const double *h_alpha, const double *d_M, const double *d_gout,
                                           double *d_out, double *d_gM, double *d_galpha, cos_stream_t stream);

/* Gradient of the determinant-weight sums from vertex coordinates (the reverse sweep of
 * cos_connected_det_matrices_grad on the gathered blocks, then the chain rule through the
 * tables as cos_connected_sum_grad):
 *   d_gM / d_gmoff  NULL, or dLoss/dM written at d_gmoff[c] as [2][n_c][n_c] (both spin
 *                   blocks, also for collapsed tables, where the blocks are equal);
 *   d_gmu           NULL or [n_cfg][2]: dLoss/dmu_b = sum_ij dLoss/dM^b_ij dM^b_ij/dmu_b; for
 *                   collapsed tables the derivative of the common matrix (the two blocks'
 *                   sum) split evenly over the two spins;
 *   d_galpha        NULL or [n_cfg][2]: dLoss/dalpha_b of the diagonal shifts h_alpha
 *                   (= -trace of dLoss/dM_b).
 * Other arguments as cos_connected_det_batch; FP64 only; builds the dG0/dmu table on first use
 * when d_gmu is given. */
cos_status cos_connected_det_grad(const cos_tables *tables, int n_cfg, int n_max, const int32_t *d_order,
                                  const int64_t *d_offset, const int32_t *d_site, const double *d_tau,
                                  const double *h_alpha, const double *d_gout, double *d_out, double *d_gM,
                                  const int64_t *d_gmoff, double *d_gmu, double *d_galpha, cos_stream_t stream);

/* Every vertex subset (the all-subsets mode of cos_connected_sum_subsets for determinant
 * weights): d_c[c * 2^n_max + S] = c(S), the connected part of det(A_up[S]) det(A_dn[S]) (the
 * close of the Alg. 1 sweep at the mask 2 1_S, rooted at min S); with d_a, a(S) =
 * det(A_up[S]) det(A_dn[S]) by the subset exponential.  Layout, all_roots, workspace and
 * errors as cos_connected_sum_subsets; h_alpha as cos_connected_det_matrices; COS_FP64 only. */
cos_status cos_connected_det_subsets(int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                                     const double *h_alpha, const double *d_M, cos_precision precision,
                                     int all_roots, double *d_c, double *d_a, cos_stream_t stream);

/* Bipartite lattice (Alg. 1 as stated): d_M4 per configuration [2][2 n_c][2 n_c] (spin block,
 * then the layout of cos_gather_bipartite), h_alpha2 = NULL or host [2][2] diagonal shifts per
 * (spin, sublattice); n_max <= COS_BIP_NMAX; precision COS_FP64, COS_MIXED or COS_DF64.  Outputs and
 * errors as cos_connected_sum_bipartite_matrices. */
cos_status cos_connected_det_bipartite_matrices(int n_cfg, int n_max, const int32_t *d_order,
                                                const int64_t *d_moff, const double *h_alpha2,
                                                const double *d_M4, cos_precision precision,
                                                double *d_out, double *d_abs_mass, cos_stream_t stream);

/* Gradient of the bipartite sums from vertex coordinates (honeycomb tables): gather, the
 * reverse sweep of cos_connected_sum_bipartite_matrices_grad, then the chain rule through
 * the tables (no counterpart in the paper, which computes no gradients):
 *   dc/dmu_l    = sum over (i,s),(j,t) of dc/dM4_l[(i,s)][(j,t)] dG_l^{st}/dmu (the gather's
 *                 interpolation of a dG/dmu table: the same 2 x 2 matrix function with
 *                 f(E) = exp(-E tau)(1 - n_F(E)) replaced by its mu derivative), G depending
 *                 on mu_l - alpha_l;
 *   dc/dalpha_l = -(that sum) + (dc/dsigma_{l,A} + dc/dsigma_{l,B}) / U, sigma_{l,A/B} =
 *                 (alpha_l +- delta_l) / U.
 * For collapsed (symmetric) tables the common derivative is split evenly over the flavors.
 * d_gM4 / d_gmoff: NULL, or dLoss/dM4 written at d_gmoff[c] as [n_mat][2 n_c][2 n_c].
 * d_gmu, d_galpha: NULL or [n_cfg][n_flavors] (per configuration, scaled by d_gout[c]).
 * Builds the dG/dmu table on first use (synchronizing `stream`).  Other arguments, limits
 * and errors as cos_connected_sum_bipartite_batch and
 * cos_connected_sum_bipartite_matrices_grad; FP64. */
cos_status cos_connected_sum_bipartite_grad(const cos_tables *tables, int n_cfg, int n_max,
                                            const int32_t *d_order, const int64_t *d_offset,
                                            const int32_t *d_site, const double *d_tau, const double *d_gout,
                                            double *d_out, double *d_gM4, const int64_t *d_gmoff,
                                            double *d_gmu, double *d_galpha, cos_stream_t stream);

/* Gather + bipartite determinant-weight sweep from vertex coordinates: two-flavor (spin up,
 * spin down) honeycomb tables of cos_build_propagators_honeycomb (tables collapsed to one
 * matrix for equal spins serve both blocks); the diagonal shifts of the determinant weights
 * are h_alpha2 (NULL or host [2][2], spin then sublattice), not the tables' shift weights.
 * Other arguments as cos_connected_sum_bipartite_batch and cos_connected_det_bipartite_matrices;
 * COS_ERR_ARG for tables with another flavor count. */
cos_status cos_connected_det_bipartite_batch(const cos_tables *tables, int n_cfg, int n_max,
                                             const int32_t *d_order, const int64_t *d_offset,
                                             const int32_t *d_site, const double *d_tau,
                                             const double *h_alpha2, cos_precision precision,
                                             double *d_out, double *d_abs_mass, cos_stream_t stream);

/* Gradient of the bipartite determinant-weight sums (the adjoint of the Alg. 1 sweep):
 * d_galpha2 NULL or [n_cfg][2][2] dLoss/dalpha_{b,s} (= minus the sublattice-s trace of
 * dLoss/dM4_b); other outputs and limits as cos_connected_sum_bipartite_matrices_grad; FP64. */
cos_status cos_connected_det_bipartite_matrices_grad(int n_cfg, int n_max, const int32_t *d_order,
                                                     const int64_t *d_moff, const double *h_alpha2,
                                                     const double *d_M4, const double *d_gout, double *d_out,
                                                     double *d_gM4, double *d_galpha2, cos_stream_t stream);

/* Gradient of the bipartite determinant-weight sums from vertex coordinates (no counterpart
 * in the paper, which computes no gradients): the gather of cos_connected_det_bipartite_batch,
 * the reverse sweep of cos_connected_det_bipartite_matrices_grad, then the chain rule through
 * the honeycomb tables as cos_connected_sum_bipartite_grad:
 *   d_gM4 / d_gmoff  NULL, or dLoss/dM4 written at d_gmoff[c] as [2][2 n_c][2 n_c] (both spin
 *                    blocks, also for collapsed tables, where the blocks are equal);
 *   d_gmu            NULL or [n_cfg][2]: dLoss/dmu_b; for collapsed tables the derivative of
 *                    the common matrix (the blocks' sum) split evenly over the two spins;
 *   d_galpha2        NULL or [n_cfg][2][2]: dLoss/dalpha_{b,s} of the diagonal shifts h_alpha2
 *                    (= minus the sublattice-s trace of dLoss/dM4_b).
 * Builds the dG/dmu table on first use when d_gmu is given (synchronizing `stream`).  Other
 * arguments and errors as cos_connected_det_bipartite_batch; FP64. */
cos_status cos_connected_det_bipartite_grad(const cos_tables *tables, int n_cfg, int n_max,
                                            const int32_t *d_order, const int64_t *d_offset,
                                            const int32_t *d_site, const double *d_tau, const double *h_alpha2,
                                            const double *d_gout, double *d_out, double *d_gM4,
                                            const int64_t *d_gmoff, double *d_gmu, double *d_galpha2,
                                            cos_stream_t stream);

/* Every vertex subset of the bipartite determinant-weight sums: d_c[c * 2^n_max + S] = c(S),
 * the connected part of sum_s det(A_up[S,s]) det(A_dn[S,s]) over the sublattice assignments s
 * of S (the close of the Alg. 1 sweep at the mask with S fully visited), and with d_a, a(S)
 * itself by the subset exponential.  d_M4 / h_alpha2 as cos_connected_det_bipartite_matrices;
 * everything else as cos_connected_sum_bipartite_subsets. */
cos_status cos_connected_det_bipartite_subsets(int n_cfg, int n_max, const int32_t *d_order,
                                               const int64_t *d_moff, const double *h_alpha2,
                                               const double *d_M4, cos_precision precision, int all_roots,
                                               double *d_c, double *d_a, cos_stream_t stream);

/* ------------------------------------------------------------------ adjoint DP
 * Gradient of the connected sums by the reverse (adjoint) DP: the forward DP is re-run with
 * every layer kept, then walked backwards (the adjoint of Alg. 2-3 as merged in Results A).
 * d_gout[c]   dLoss/dc for configuration c (the vector the gradient is contracted with)
 * d_out       NULL or receives c (as cos_connected_sum_matrices, FP64)
 * d_gM        NULL or receives dLoss/dM, same layout and offsets (d_moff) as d_M
 * d_gsigma    NULL or receives dLoss/dsigma_l per configuration, [n_cfg][n_mat] (computed
 *             also at sigma = 0, where shift transitions carry no weight)
 * Other arguments as cos_connected_sum_matrices.  FP64 only. */
cos_status cos_connected_sum_matrices_grad(int n_cfg, int n_max, const int32_t *d_order,
                                           const int64_t *d_moff, int n_mat, int loop_weight,
                                           const double *h_sigma, const double *d_M,
                                           const double *d_gout, double *d_out, double *d_gM,
                                           double *d_gsigma, cos_stream_t stream);

/* Memory of the gradient calls.  The reverse sweep needs the forward state of every layer;
 * each adjoint overwrites the forward state it was formed from, so the kept layers are the
 * whole workspace: about (states per flavor array) x 32 lanes x 8 B per CTA, 181 MB at n = 10
 * and 2.2 GB at n = 12.  Where free device memory cannot hold that for every CTA, layers are
 * checkpointed (the reverse of Alg. 2-3 with the forward recomputed per segment): a set of
 * checkpoint layers is kept, and the layers between two checkpoints are re-run from the first
 * before they are reversed.  The launcher picks, per order, the grid and checkpoint set that
 * give the most throughput within 85 % of the free memory.  The environment variable
 * COS_GRAD_CHECKPOINT=1 forces the least-storage plan at every order, =0 keeps every layer.
 *
 * cos_grad_checkpoint_plan (host only, no device): the plan of order n for a budget of
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
 * configuration): warps per CTA (1..16), resident CTAs per SM (1..8) and whether a warp
 * prefetches the states of its next mask while it computes the current one (prefetch:
 * 0 = off, 1 = into L2, 2 = into L1).  A launch mixing
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
