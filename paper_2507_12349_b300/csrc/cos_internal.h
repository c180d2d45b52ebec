// Internal declarations of libcos (CUDA side).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "cos.h"

namespace cosdp {

constexpr int kLanes = 32;          // lanes of a warp = (configuration, flavor) pairs of a batch
constexpr int kMaxLayers = 2 * COS_NMAX + 1;

// Device status bits (OR-ed into the per-stream status word).
enum : int {
    kStatusOrder = 1,
    kStatusSite = 2,
    kStatusNonFinite = 4,
};

// One interaction mask mu in {0,1,2}^n with mu_0 >= 1, as stored on the device.
//   ab   : visited set A = {i : mu_i >= 1} in bits 0..15, full set B = {i : mu_i = 2} in bits 16..31
//   code : sum_i mu_i 3^i
//   off  : offset (in state slots) of the mask's block inside its layer; the block holds
//          |H(mu)| rows (heads) of |A| slots (endpoints), slot (h, v) at off + idxH(h)*|A| + idxA(v)
struct MaskRec {
    uint32_t ab;
    uint32_t code;
    uint32_t off;
    uint32_t cost;
};

// Structure of the merged DP for one order n, device copy.
struct OrderTab {
    const MaskRec *masks;     // grouped by layer, cost-sorted (descending) inside a layer
    const uint32_t *rank3;    // code -> block offset inside its layer
    const uint32_t *ord3;     // code -> ordinal of the mask inside its layer (null where unused)
    uint32_t layer_first[kMaxLayers + 1];
    uint32_t layer_count[kMaxLayers + 1];
    uint32_t layer_slots[kMaxLayers + 1];
    uint32_t max_slots;
    uint32_t max_masks;       // most masks in one layer
    uint32_t n;
};

// Endpoints v that a row (mu, h) can hold (reachable slots; the others are never written
// and never read).  A = visited set, ones = {i : mu_i = 1}.
//   h = 0, mu_0 = 1 : the first loop has visited only point 0 of vertex 0, so v = 0 only at the
//                     start mu = e_0; otherwise v ranges over A \ {0}.
//   h = 0, mu_0 = 2 : every visited vertex.
//   h != 0          : later loops never return to vertex 0 (it was full before they opened);
//                     v = h only if h was the smallest half-visited vertex when the loop opened,
//                     i.e. no vertex below h is half-visited now.
__host__ __device__ inline uint32_t row_vmask(uint32_t A, uint32_t ones, int h) {
    if (h == 0) {
        if (ones & 1u) return (A == 1u) ? 1u : (A & ~1u);
        return A;
    }
    uint32_t v = A & ~1u;
    if (ones & ((1u << h) - 1u)) v &= ~(1u << h);
    return v;
}

// Heads of the open loop: vertex 0 while the first loop is open with mu_0 = 1, else the full set.
__host__ __device__ inline uint32_t head_set(uint32_t B, uint32_t ones) {
    return (ones & 1u) ? 1u : B;
}

// Host-side structure (built once per order).
struct HostOrder {
    int n = 0;
    std::vector<MaskRec> masks;
    std::vector<uint32_t> rank3;
    std::vector<uint32_t> ord3;
    uint32_t layer_first[kMaxLayers + 1] = {};
    uint32_t layer_count[kMaxLayers + 1] = {};
    uint32_t layer_slots[kMaxLayers + 1] = {};
    uint32_t max_slots = 0;
    uint32_t max_masks = 0;
    uint64_t layer_work[kMaxLayers + 1] = {};   // multiply-adds of the sweep out of each layer (one flavor array)
    cos_structure_info info{};
};

const HostOrder &host_order(int n);   // thread-safe, cached

// Per-device copy of the tables of orders 1..COS_NMAX; returns a device array of 13 OrderTab.
const OrderTab *device_orders(int device, std::string *err);

// Thread-local error message.
void set_error(const std::string &msg);
cos_status cuda_fail(cudaError_t e, const char *what);

// Per (device, stream) workspace.
struct Workspace {
    int device = -1;
    cudaStream_t stream = nullptr;
    int *status = nullptr;           // device status word
    // planner
    int *plan_counts = nullptr;      // [16] counts per order, [16] cursors, [16] bucket starts, [16] batch starts, [4] misc
    int *batch_list = nullptr;       // sorted configuration indices
    int4 *batches = nullptr;         // {n, start, count, 0}
    size_t batches_cap = 0;          // capacity in batches
    size_t batch_cap = 0;            // capacity in configurations
    int *queue = nullptr;            // persistent-kernel work counter
    // gathered matrices (batch path)
    double *M = nullptr;
    size_t M_cap = 0;                // doubles
    int64_t *moff = nullptr;
    size_t moff_cap = 0;
    // DP layer scratch
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    // all-subsets mode: derived suffix problems (order, matrix offset, output key) and matrices
    int32_t *sub_order = nullptr;
    int64_t *sub_moff = nullptr;
    int64_t *sub_key = nullptr;
    size_t sub_cap = 0;              // derived problems (each of the three arrays)
    size_t sub_moff_cap = 0;
    size_t sub_key_cap = 0;
    double *sub_M = nullptr;
    size_t sub_M_cap = 0;            // doubles
    // gradient path
    double *gM = nullptr;
    size_t gM_cap = 0;
    double *gsig = nullptr;
    size_t gsig_cap = 0;
    // launch shape: fixed_grid > 0 pins the persistent grid (plans captured in a graph);
    // last_grid records the grid of the latest DP launch.
    int fixed_grid = 0;
    int last_grid = 0;
};

Workspace *get_workspace(cudaStream_t stream, std::string *err);
cos_status ensure(void **ptr, size_t *cap, size_t need, size_t elem, const char *what);

// Launch tuning for one order.
struct Tuning {
    int warps = 8;          // warps per CTA
    int ctas_per_sm = 2;    // resident CTAs per SM targeted by the persistent grid
    int prefetch = 1;       // prefetch the next mask's states: 0 off, 1 into L2, 2 into L1
};
Tuning get_tuning(int n, int precision, int nf_lanes);
void set_tuning(int n, int precision, int nf_lanes, Tuning t);
Workspace *new_private_workspace(int device, std::string *err);   // not registered per stream
void free_workspace(Workspace *ws);

struct DpLaunch {
    int n_cfg = 0;
    int n_max = 0;
    const int32_t *order = nullptr;
    const double *M = nullptr;
    const int64_t *moff = nullptr;
    int64_t mstride = 0;            // used when moff == nullptr
    int n_mat = 1;
    int loop_weight = 1;
    double sigma[COS_MAX_FLAVORS] = {};
    bool shifts = false;
    int precision = COS_FP64;
    double *out = nullptr;
    bool absmode = false;
    double *csub = nullptr;         // all-subsets mode: c(S) written at csub[base + (S << shift)]
    const int64_t *csub_key = nullptr;  // per configuration: (base << 4) | shift
    bool allow_empty = false;       // order 0 = empty configuration slot (skipped by the planner)
    bool clow = false;              // determinant weights without cycle factors (two spin blocks)
};

cos_status launch_plan_batches(Workspace *ws, int n_cfg, int n_max, const int32_t *order, int cpb,
                               cudaStream_t stream, bool allow_empty = false);
cos_status launch_dp(Workspace *ws, const DpLaunch &a, cudaStream_t stream);
// Launch the planner and the DP kernel on caller-provided device buffers (no allocation):
// plan = 80 ints, queue = 1 int, status = 1 int, list = n_cfg ints, batches = max_batches int4,
// scratch = grid * nslots * slot_elems elements of the state type, tabs = device OrderTab[13].
struct RawBuffers {
    int *plan;
    int *queue;
    int *status;
    int *list;
    int4 *batches;
    void *scratch;
    const OrderTab *tabs;
    int grid;
};
cos_status launch_plan_raw(const RawBuffers &rb, int n_cfg, int n_max, const int32_t *order, int cpb, int device,
                           cudaStream_t stream);
cos_status launch_dp_raw(const RawBuffers &rb, const DpLaunch &a, cudaStream_t stream);
int dp_slots(const DpLaunch &a);            // layer slots of the ring: always 2 (shifts ride on the diagonal)
// Mixed and double-float precision run two configurations per lane (cos_dp_pair.cu) except
// in the all-subsets mode; configurations per batch follow the kernel the launch selects.
bool dp_uses_pair(const DpLaunch &a);
int dp_configs_per_batch(const DpLaunch &a);
cos_status launch_dp_pair(Workspace *ws, const DpLaunch &a, cudaStream_t stream);
size_t pair_smem_bytes(int precision, int n_max);
int pair_width(int precision);   // configurations per lane of the pair kernel of a precision
int pair_max_active_ctas(int precision, int threads, size_t smem);
size_t dp_smem_bytes(int precision, int n_max);   // forward kernel shared memory of a precision
size_t dp_state_bytes(const DpLaunch &a);   // bytes per state element

// Checkpoint plans of the gradients' kept layers (cos_adjoint.cu): a set of checkpoint layers
// (bit l of mask), the slots per lane it keeps (checkpoints + the largest segment interior) and
// the multiply-adds of one flavor array it re-runs; lattice COS_SQUARE or COS_BIPARTITE.
struct CkPlan {
    uint32_t mask = 0;
    uint64_t store = 0;
    uint64_t recompute = 0;
    bool ok = false;
};
CkPlan ck_plan(int lattice, int n, uint64_t budget);   // least recomputation within budget (0: least storage)
CkPlan ck_full(int lattice, int n);                    // every layer kept
uint64_t ck_forward_work(int lattice, int n);          // multiply-adds of one forward sweep
int checkpoint_mode();                                  // COS_GRAD_CHECKPOINT: -1 unset, 0 keep all, 1 least storage
void bip_layer_profile(int n, uint64_t *slots, uint64_t *work);   // per-layer slots / work, bipartite

cos_status launch_adjoint(Workspace *ws, const DpLaunch &a, const double *gout, double *gM, const int64_t *gmoff,
                          int64_t gmstride, double *gsig, cudaStream_t stream);
cos_status launch_chain(const cos_tables *t, int n_cfg, const int32_t *order, const int64_t *offset,
                        const int32_t *site, const double *tau, const double *gM, const int64_t *gmoff,
                        int64_t gmstride, const double *gsig, double *gmu, double *galpha, cudaStream_t stream);
cos_status ensure_dtables(cos_tables *t, cudaStream_t stream);

cos_status check_common(int n_cfg, int n_max, cos_precision prec, const char *fn);
cos_status run_dp(Workspace *ws, DpLaunch L, double *d_abs_mass, cudaStream_t stream);
cos_status matrices_body(Workspace *ws, int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                         int n_mat, int loop_weight, const double *h_sigma, const double *d_M,
                         cos_precision precision, double *d_out, double *d_abs_mass, cudaStream_t stream);
cos_status check_matrices(int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff, int n_mat,
                          int loop_weight, const double *d_M, cos_precision precision, const double *d_out,
                          const char *fn);
cos_status check_batch(const cos_tables *t, int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_offset,
                       const int32_t *d_site, const double *d_tau, cos_precision precision, const double *d_out,
                       const char *fn);
cos_status batch_body(Workspace *ws, const cos_tables *t, int n_cfg, int n_max, const int32_t *d_order,
                      const int64_t *d_offset, const int32_t *d_site, const double *d_tau, cos_precision precision,
                      double *d_out, double *d_abs_mass, cudaStream_t stream);
int dp_max_active_ctas(int precision, int threads, size_t smem);

cos_status bip_matrices_body(Workspace *ws, int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                             int n_mat, int loop_weight, const double *h_sigma2, const double *d_M4,
                             cos_precision precision, double *d_out, double *d_abs_mass, cudaStream_t stream,
                             bool clow = false);
// Bipartite reverse sweep (FP64) on matrices at d_moff; dc/dM4 at the same offsets.  clow:
// determinant weights (n_mat = 2 spin blocks, h_sigma2 = the diagonal shifts alpha2).
cos_status bip_grad_dp(const char *fn, int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                       int n_mat, int loop_weight, const double *h_sigma2, const double *d_M4, const double *d_gout,
                       double *d_out, double *d_gM4, double *d_gsigma2, cudaStream_t stream, bool clow = false);
// Bipartite sweep in the all-subsets mode (FP64): planner (allow_empty: order-0 derived
// problems skipped) + DP, c(S) written through d_csub / d_csub_key.
cos_status bip_subsets_dp(Workspace *ws, int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                          int n_mat, int loop_weight, const double *h_sigma2, const double *d_M4, bool clow,
                          double *d_csub, const int64_t *d_csub_key, bool allow_empty, cudaStream_t stream);

cos_status launch_gather(const cos_tables *t, int n_cfg, const int32_t *order, const int64_t *offset,
                         const int32_t *site, const double *tau, const int64_t *moff, int64_t mstride,
                         double *M, int *status, cudaStream_t stream);

}  // namespace cosdp

struct cos_tables {
    int device;
    cos_model model;          // mu/alpha point into the vectors below
    std::vector<double> mu, alpha;
    int n_mat;
    int symmetric;
    double sigma[COS_MAX_FLAVORS];
    double *d_G;              // square: [n_mat][L^2][n_tau]; honeycomb: [n_mat][2][2][L^2][n_tau]
    double *d_dG;
    int bipartite = 0;        // honeycomb (two-band) tables
    std::vector<double> delta;
    double sigma2[COS_MAX_FLAVORS][2] = {};   // honeycomb: shift weight per (flavor, sublattice)
};

// The per-case implementations behind cos_forward, cos_grad and cos_subsets (cos_api.cu): one
// per lattice, weight kind and input form.  C linkage, hidden from the library's exports; the
// public header documents their arguments through cos_problem.
#define COS_INTERNAL_API extern "C" __attribute__((visibility("hidden")))
COS_INTERNAL_API cos_status cos_connected_sum_subsets(int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                                     int n_mat, int loop_weight, const double *h_sigma, const double *d_M,
                                     cos_precision precision, int all_roots, double *d_c, double *d_a,
                                     cos_stream_t stream);
COS_INTERNAL_API cos_status cos_connected_sum_bipartite_matrices(int n_cfg, int n_max, const int32_t *d_order,
                                                const int64_t *d_moff, int n_mat, int loop_weight,
                                                const double *h_sigma2, const double *d_M4,
                                                cos_precision precision, double *d_out,
                                                double *d_abs_mass, cos_stream_t stream);
COS_INTERNAL_API cos_status cos_connected_sum_bipartite_matrices_grad(int n_cfg, int n_max, const int32_t *d_order,
                                                     const int64_t *d_moff, int n_mat, int loop_weight,
                                                     const double *h_sigma2, const double *d_M4, const double *d_gout,
                                                     double *d_out, double *d_gM4, double *d_gsigma2,
                                                     cos_stream_t stream);
COS_INTERNAL_API cos_status cos_connected_sum_bipartite_batch(const cos_tables *tables, int n_cfg, int n_max,
                                             const int32_t *d_order, const int64_t *d_offset,
                                             const int32_t *d_site, const double *d_tau,
                                             cos_precision precision, double *d_out,
                                             double *d_abs_mass, cos_stream_t stream);
COS_INTERNAL_API cos_status cos_connected_sum_bipartite_subsets(int n_cfg, int n_max, const int32_t *d_order,
                                               const int64_t *d_moff, int n_mat, int loop_weight,
                                               const double *h_sigma2, const double *d_M4,
                                               cos_precision precision, int all_roots, double *d_c,
                                               double *d_a, cos_stream_t stream);
COS_INTERNAL_API cos_status cos_connected_det_matrices(int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                                      const double *h_alpha, const double *d_M, cos_precision precision,
                                      double *d_out, double *d_abs_mass, cos_stream_t stream);
COS_INTERNAL_API cos_status cos_connected_det_batch(const cos_tables *tables, int n_cfg, int n_max, const int32_t *d_order,
                                   const int64_t *d_offset, const int32_t *d_site, const double *d_tau,
                                   const double *h_alpha, cos_precision precision, double *d_out,
                                   double *d_abs_mass, cos_stream_t stream);
COS_INTERNAL_API cos_status cos_connected_det_matrices_grad(int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                                           const double *h_alpha, const double *d_M, const double *d_gout,
                                           double *d_out, double *d_gM, double *d_galpha, cos_stream_t stream);
COS_INTERNAL_API cos_status cos_connected_det_grad(const cos_tables *tables, int n_cfg, int n_max, const int32_t *d_order,
                                  const int64_t *d_offset, const int32_t *d_site, const double *d_tau,
                                  const double *h_alpha, const double *d_gout, double *d_out, double *d_gM,
                                  const int64_t *d_gmoff, double *d_gmu, double *d_galpha, cos_stream_t stream);
COS_INTERNAL_API cos_status cos_connected_det_subsets(int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                                     const double *h_alpha, const double *d_M, cos_precision precision,
                                     int all_roots, double *d_c, double *d_a, cos_stream_t stream);
COS_INTERNAL_API cos_status cos_connected_det_bipartite_matrices(int n_cfg, int n_max, const int32_t *d_order,
                                                const int64_t *d_moff, const double *h_alpha2,
                                                const double *d_M4, cos_precision precision,
                                                double *d_out, double *d_abs_mass, cos_stream_t stream);
COS_INTERNAL_API cos_status cos_connected_sum_bipartite_grad(const cos_tables *tables, int n_cfg, int n_max,
                                            const int32_t *d_order, const int64_t *d_offset,
                                            const int32_t *d_site, const double *d_tau, const double *d_gout,
                                            double *d_out, double *d_gM4, const int64_t *d_gmoff,
                                            double *d_gmu, double *d_galpha, cos_stream_t stream);
COS_INTERNAL_API cos_status cos_connected_det_bipartite_batch(const cos_tables *tables, int n_cfg, int n_max,
                                             const int32_t *d_order, const int64_t *d_offset,
                                             const int32_t *d_site, const double *d_tau,
                                             const double *h_alpha2, cos_precision precision,
                                             double *d_out, double *d_abs_mass, cos_stream_t stream);
COS_INTERNAL_API cos_status cos_connected_det_bipartite_matrices_grad(int n_cfg, int n_max, const int32_t *d_order,
                                                     const int64_t *d_moff, const double *h_alpha2,
                                                     const double *d_M4, const double *d_gout, double *d_out,
                                                     double *d_gM4, double *d_galpha2, cos_stream_t stream);
COS_INTERNAL_API cos_status cos_connected_det_bipartite_grad(const cos_tables *tables, int n_cfg, int n_max,
                                            const int32_t *d_order, const int64_t *d_offset,
                                            const int32_t *d_site, const double *d_tau, const double *h_alpha2,
                                            const double *d_gout, double *d_out, double *d_gM4,
                                            const int64_t *d_gmoff, double *d_gmu, double *d_galpha2,
                                            cos_stream_t stream);
COS_INTERNAL_API cos_status cos_connected_det_bipartite_subsets(int n_cfg, int n_max, const int32_t *d_order,
                                               const int64_t *d_moff, const double *h_alpha2,
                                               const double *d_M4, cos_precision precision, int all_roots,
                                               double *d_c, double *d_a, cos_stream_t stream);
COS_INTERNAL_API cos_status cos_connected_sum_matrices_grad(int n_cfg, int n_max, const int32_t *d_order,
                                           const int64_t *d_moff, int n_mat, int loop_weight,
                                           const double *h_sigma, const double *d_M,
                                           const double *d_gout, double *d_out, double *d_gM,
                                           double *d_gsigma, cos_stream_t stream);
