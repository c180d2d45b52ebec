// K-DP: the merged clow-sequence dynamic program (Results A, Alg. 2-3) on sm_103a.
//
// Work decomposition
//   * A batch is up to 32 (configuration, flavor) pairs of one order n: lane = c * nf_lanes + l.
//     Every lane runs the same structural schedule, so control flow is warp-uniform and every
//     state / matrix access of a warp is one coalesced 256-byte (FP64) row.
//   * One CTA owns a batch.  Its warps split the interaction masks of each layer (cost-sorted
//     round robin); layers are separated by __syncthreads.  Persistent CTAs pull batches from a
//     queue ordered by decreasing order n (largest work first).
//   * The batch's matrices sit in shared memory as [v][j][lane]; layer states live in a per-CTA
//     global ring of 2 layer slots laid out [slot][lane].
//
// Recurrence (push form, per row = mask mu, head h, lane flavor l, endpoints v in Vrow):
//   close   csum(mu)            += sum_v O(mu,h,v) Md[v][h]     Md = sgn w M   (Alg. 2 Close)
//   extend  O(mu+e_j, h, j)      = d_j = sum_v O(mu,h,v) Ms[v][j], mu_j <= 1    (Alg. 2 Extend)
//   after all rows of mu:  C(mu) = sum over the lanes of the configuration of csum (flavor sum)
//            mu has a 1 -> O(mu+e_k, k, k) = C(mu) in every flavor, k = min{i: mu_i = 1}
//            mu full    -> c = 2^(n-1) C(mu)
// The factor 2 for entering an untouched vertex (either of its two points) is the same on
// every path -- each vertex other than 0 is entered from mu_j = 0 exactly once -- so it is
// pulled out as the global 2^(n-1); the start with a shifted vertex 0 keeps its 2 (-2 sigma).
//
// Shift points (Alg. 3: a shift takes the color of its partner's loop and closes at once with
// -sigma).  Entering an untouched vertex j whose other point is a shift gives the state
// (mu + 2e_j, h, j) the weight -sigma d_j, where d_j is the very value the same extension
// stores at (mu + e_j, h, j) -- that slot's only writer.  So the shift contribution is
// -sigma O(mu+e_j, h, j), taken when the row (mu + e_j, h) extends from endpoint j into the
// other point of j: the extension matrix carries Ms[j][j] = M[j][j] - sigma for j >= 1 (the
// close keeps the unshifted diagonal, vertex 0 keeps its start seed).  Every target slot has
// a single writer, the ring needs two layer slots, and slots never need clearing between
// batches (each one read in a batch is written earlier in that batch).
//
// Determinant weights without cycle factors (Results A, Alg. 1; CLOW instantiations).  For an
// SU(2) model with the interaction n_up n_dn every vertex has a spin-up point (block 0) and a
// spin-down point (block 1), and the matrix is block diagonal in spin.  Alg. 1 keeps only the
// interaction mask, so a clow may visit one point twice; those nonphysical sequences cancel.
// A point is (vertex, block), so the state ((u), (v), mu) of Alg. 1 is the merged state
// (mu, h, v) in the lane of block b, and the sweep above applies with four changes: entering
// an untouched vertex has weight 1 (no 2^(n-1)); the start is in block 0 only; the first loop
// (head point 0 of block 0) never steps onto vertex 0; and its close opens the next loop at
// the other point of vertex 0, i.e. in block 1 only.  Every other close opens at both points
// of vertex k, one per block, which is the flavor-sum seed.  Diagonal shifts alpha_b of the
// density (n_b - alpha_b) enter both matrix copies, the close's included.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "cos_dp_device.cuh"

namespace cosdp {

// State type -> close-matrix type (converted from the FP64 inputs once per batch): FP64 for
// FP64 states, FP32 pairs for FP32 states (the mixed mode's compensated close) and df64 states.
template <typename T>
struct CloseOf {
    using type = double;
};
template <>
struct CloseOf<float> {
    using type = df64;
};
template <>
struct CloseOf<df64> {
    using type = df64;
};

// Register budgets: MAXT = 256 (two CTAs of up to 8 warps, <= 128 registers), MAXT = 320 (FP64:
// two CTAs of up to 10 warps, <= 96 registers), MAXT = 384 (up to 12 warps; FP32 two CTAs, <= 85
// registers) and MAXT = 512 (up to 16 warps; <= 128 registers in FP64 with one CTA, <= 64 in FP32
// with two).
// SUB: all-subsets mode (closes of masks with no half-visited vertex stored through csub_key).
// CLOW: determinant weights without cycle factors (two spin-block lanes per configuration).
template <typename T, int MAXT, bool SUB, bool CLOW = false>
__global__ void __launch_bounds__(MAXT, (MAXT <= 320 || sizeof(T) == 4) ? 2 : 1)
    dp_forward_kernel(const __grid_constant__ DpArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_batch;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int nsm = a.smem_n * a.smem_n * kLanes;
    // Ms: matrices for the extension (state type); Md: FP64 matrices times the loop factor
    // sgn * w for the close (so the close needs no extra multiply per mask).
    using CT = typename CloseOf<T>::type;
    constexpr bool kDf = std::is_same<T, df64>::value;
    T *Ms = reinterpret_cast<T *>(smem_raw);
    CT *Mdw = reinterpret_cast<CT *>(smem_raw + ((nsm * sizeof(T) + 15) & ~size_t(15)));
    const CT *Md = Mdw;
    T *ring = reinterpret_cast<T *>(a.scratch) + (size_t)blockIdx.x * a.nslots * a.slot_elems;
    const int nfl = a.nf_lanes;
    const int lam = lane % nfl;
    const int ci = lane / nfl;
    const double sgn = a.absmode ? 1.0 : -1.0;
    const double sig = a.absmode ? fabs(a.sigma[lam]) : a.sigma[lam];
    const bool shifts = a.shifts != 0;
    const int nbatch = *a.n_batches;
    df64 seed0 = {0.0f, 0.0f};
    if (kDf) seed0 = df64_from(sgn * 2.0 * sig);

    for (;;) {
        __syncthreads();  // previous batch fully done before s_batch / smem are reused
        if (threadIdx.x == 0) s_batch = atomicAdd(a.queue, 1);
        __syncthreads();
        const int b = s_batch;
        if (b >= nbatch) break;
        const int4 bd = a.batches[b];
        const int n = bd.x;
        const OrderTab &tab = a.tabs[n];
        const bool active = (ci < bd.z) && (ci * nfl + nfl <= kLanes);
        const int cfg = active ? a.batch_list[bd.y + ci] : -1;
        const double *Mc = nullptr;
        if (active) Mc = a.M + (a.moff ? a.moff[cfg] : (int64_t)cfg * a.mstride) + (size_t)lam * n * n;
        double *cs = nullptr;
        int csh = 0;
        if (SUB && active) {
            const int64_t key = a.csub_key[cfg];
            cs = a.csub + (key >> 4);
            csh = (int)(key & 15);
        }
        // Matrices of the batch -> shared memory [v][j][lane].
        const double cfac = sgn * a.loop_weight;
        const double dshift = sgn * sig;   // -sigma (|sigma| for the mass)
        for (int e = warp; e < n * n; e += nwarps) {
            double val = active ? Mc[e] : 0.0;
            if (a.absmode) val = fabs(val);
            const int v = e / n, j = e % n;
            if (CLOW) {
                const double m = (v == j) ? val + dshift : val;   // a(p, p) - alpha_b everywhere
                to_elem(m, Ms[e * kLanes + lane]);
                to_elem(cfac * m, Mdw[e * kLanes + lane]);
            } else {
                to_elem((v == j && j != 0 && shifts) ? val + dshift : val, Ms[e * kLanes + lane]);
                to_elem(cfac * val, Mdw[e * kLanes + lane]);
            }
        }
        // Start: the loop through the normal point of vertex 0 (layer 1, mask e_0, slot 0);
        // determinant weights start at the spin-up point only.
        if (warp == 0) to_elem((CLOW && lam != 0) ? 0.0 : 1.0, ring[(1 % a.nslots) * a.slot_elems + lane]);
        __syncthreads();

        for (int ell = 1; ell <= 2 * n; ++ell) {
            const T *src = ring + (size_t)(ell % a.nslots) * a.slot_elems;
            T *dst1 = ring + (size_t)((ell + 1) % a.nslots) * a.slot_elems;
            const uint32_t first = tab.layer_first[ell];
            const uint32_t cnt = tab.layer_count[ell];
            for (uint32_t mi = warp; mi < cnt; mi += nwarps) {
                const uint32_t next = mi + nwarps < cnt ? first + mi + nwarps : 0xFFFFFFFFu;
                if constexpr (kDf)
                    fwd_mask_df<SUB>(tab, first + mi, next, ell, n, src, dst1, Ms, Md, lane, ci, nfl, seed0, shifts,
                                     active, lam, cfg, a.out, a.status, a.prefetch, cs, csh);
                else
                    fwd_mask<T, SUB, CLOW, CT>(tab, first + mi, next, ell, n, src, dst1, Ms, Md, lane, ci, nfl, sgn,
                                               sig, shifts, active, lam, cfg, a.out, a.status, a.prefetch, cs, csh);
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------ batch planner
// Sorts configurations by order (largest first) into batches of `cpb` configurations.
// plan layout: [0,16) counts, [16,32) cursors, [32,48) bucket starts, [48,64) batch starts, [64] n_batches

// allow_empty: order 0 marks a configuration slot with nothing to compute (derived problems of
// the all-subsets mode); it is skipped instead of flagged.
__global__ void plan_count_kernel(int n_cfg, int n_max, const int32_t *order, int *plan, int *status,
                                  int allow_empty) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cfg; c += gridDim.x * blockDim.x) {
        const int n = order[c];
        if (n == 0 && allow_empty) continue;
        if (n < 1 || n > n_max) {
            atomicOr(status, kStatusOrder);
        } else {
            atomicAdd(&plan[n], 1);
        }
    }
}

__global__ void plan_prefix_kernel(int cpb, int *plan) {
    if (threadIdx.x != 0) return;
    int run = 0, brun = 0;
    for (int n = COS_NMAX; n >= 1; --n) {
        plan[32 + n] = run;
        plan[48 + n] = brun;
        run += plan[n];
        brun += (plan[n] + cpb - 1) / cpb;
    }
    plan[64] = brun;
}

__global__ void plan_scatter_kernel(int n_cfg, int n_max, const int32_t *order, int *plan, int *list) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cfg; c += gridDim.x * blockDim.x) {
        const int n = order[c];
        if (n < 1 || n > n_max) continue;
        const int pos = atomicAdd(&plan[16 + n], 1);
        list[plan[32 + n] + pos] = c;
    }
}

__global__ void plan_batches_kernel(int max_batches, int cpb, const int *plan, int4 *batches) {
    const int nb = plan[64];
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < max_batches && b < nb; b += gridDim.x * blockDim.x) {
        int n = COS_NMAX;
        while (n > 1 && b >= plan[48 + n] + (plan[n] + cpb - 1) / cpb) --n;
        const int local = b - plan[48 + n];
        const int start = plan[32 + n] + local * cpb;
        const int count = min(cpb, plan[n] - local * cpb);
        batches[b] = make_int4(n, start, count, 0);
    }
}

static int sm_count(int device) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    return v > 0 ? v : 1;
}

cos_status launch_plan_batches(Workspace *ws, int n_cfg, int n_max, const int32_t *order, int cpb,
                               cudaStream_t stream, bool allow_empty) {
    const int max_batches = (n_cfg + cpb - 1) / cpb + COS_NMAX;
    cos_status st = ensure((void **)&ws->batch_list, &ws->batch_cap, (size_t)n_cfg + 1, sizeof(int), "batch list");
    if (st != COS_OK) return st;
    st = ensure((void **)&ws->batches, &ws->batches_cap, (size_t)max_batches, sizeof(int4), "batch table");
    if (st != COS_OK) return st;
    cudaError_t e = cudaMemsetAsync(ws->plan_counts, 0, 80 * sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e, "planner memset");
    const int threads = 256;
    const int blocks = std::max(1, std::min((n_cfg + threads - 1) / threads, 4 * sm_count(ws->device)));
    if (n_cfg > 0)
        plan_count_kernel<<<blocks, threads, 0, stream>>>(n_cfg, n_max, order, ws->plan_counts, ws->status,
                                                          allow_empty ? 1 : 0);
    plan_prefix_kernel<<<1, 32, 0, stream>>>(cpb, ws->plan_counts);
    if (n_cfg > 0) plan_scatter_kernel<<<blocks, threads, 0, stream>>>(n_cfg, n_max, order, ws->plan_counts, ws->batch_list);
    const int bb = std::max(1, std::min((max_batches + threads - 1) / threads, 4 * sm_count(ws->device)));
    plan_batches_kernel<<<bb, threads, 0, stream>>>(max_batches, cpb, ws->plan_counts, ws->batches);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "planner launch");
    return COS_OK;
}

template <typename T, bool SUB, bool CLOW = false>
static auto forward_kernel_for(int threads) {
    if (threads <= 256) return dp_forward_kernel<T, 256, SUB, CLOW>;
    // FP64 sweeps (every mode): two CTAs of up to 10 warps (<= 96 registers)
    if constexpr (std::is_same<T, double>::value) {
        if (threads <= 320) return dp_forward_kernel<T, 320, SUB, CLOW>;
    }
    return threads <= 384 ? dp_forward_kernel<T, 384, SUB, CLOW> : dp_forward_kernel<T, 512, SUB, CLOW>;
}

// Determinant weights (L.clow) reach this launcher in FP64 only: the reduced precisions run
// the pair kernels (cos_dp_pair.cu), and their all-subsets mode is FP64.
template <typename T>
static auto kernel_for_launch(const DpLaunch &L, int threads) {
    if constexpr (std::is_same<T, double>::value) {
        if (L.clow) return L.csub ? forward_kernel_for<T, true, true>(threads) : forward_kernel_for<T, false, true>(threads);
    }
    return L.csub ? forward_kernel_for<T, true>(threads) : forward_kernel_for<T, false>(threads);
}

template <typename T>
static cos_status launch_dp_t(Workspace *ws, const DpLaunch &L, cudaStream_t stream) {
    std::string err;
    const OrderTab *tabs = device_orders(ws->device, &err);
    if (!tabs) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    const int nfl = L.n_mat;
    const Tuning tu = get_tuning(L.n_max, L.precision, nfl);
    const int nsm = sm_count(ws->device);
    const int nslots = dp_slots(L);
    const size_t slot_elems = (size_t)host_order(L.n_max).max_slots * kLanes;
    const size_t per_cta = (size_t)nslots * slot_elems * sizeof(T);
    const int cpb = kLanes / nfl;
    const int max_batches = (L.n_cfg + cpb - 1) / cpb + COS_NMAX;
    int grid = std::max(1, std::min(nsm * tu.ctas_per_sm, max_batches));
    if (ws->fixed_grid > 0) {
        grid = ws->fixed_grid;
    } else {
        // Keep the layer scratch inside the free device memory (leave headroom for the caller).
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
            const size_t avail = ws->scratch_bytes + (size_t)(0.85 * (double)free_b);
            while (grid > 1 && (size_t)grid * per_cta > avail) grid = std::max(1, grid / 2);
        }
    }
    ws->last_grid = grid;
    cos_status st = ensure(&ws->scratch, &ws->scratch_bytes, (size_t)grid * per_cta, 1, "layer scratch");
    if (st != COS_OK) return st;
    const int threads = tu.warps * 32;
    const size_t msm = (size_t)L.n_max * L.n_max * kLanes;
    const size_t smem = ((msm * sizeof(T) + 15) & ~size_t(15)) + msm * sizeof(typename CloseOf<T>::type);
    auto kern = kernel_for_launch<T>(L, threads);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "dp smem attribute");
    DpArgs a;
    memset(&a, 0, sizeof a);
    a.tabs = tabs;
    a.batches = ws->batches;
    a.n_batches = ws->plan_counts + 64;
    a.batch_list = ws->batch_list;
    a.queue = ws->queue;
    a.M = L.M;
    a.moff = L.moff;
    a.mstride = L.mstride;
    a.nf_lanes = nfl;
    a.loop_weight = (double)L.loop_weight;
    for (int l = 0; l < COS_MAX_FLAVORS; ++l) a.sigma[l] = L.sigma[l];
    a.shifts = L.shifts ? 1 : 0;
    a.absmode = L.absmode ? 1 : 0;
    a.scratch = ws->scratch;
    a.slot_elems = slot_elems;
    a.nslots = nslots;
    a.smem_n = L.n_max;
    a.prefetch = tu.prefetch;
    a.csub = L.csub;
    a.csub_key = L.csub_key;
    a.out = L.out;
    a.status = ws->status;
    e = cudaMemsetAsync(ws->queue, 0, sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e, "queue reset");
    kern<<<grid, threads, smem, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "dp launch");
    return COS_OK;
}

// ------------------------------------------------------------------ raw-buffer launchers

int dp_slots(const DpLaunch &) { return 2; }
size_t dp_state_bytes(const DpLaunch &L) { return L.precision == COS_MIXED ? sizeof(float) : sizeof(double); }

cos_status launch_plan_raw(const RawBuffers &rb, int n_cfg, int n_max, const int32_t *order, int cpb, int device,
                           cudaStream_t stream) {
    const int max_batches = (n_cfg + cpb - 1) / cpb + COS_NMAX;
    cudaError_t e = cudaMemsetAsync(rb.plan, 0, 80 * sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e, "planner memset");
    const int threads = 256;
    const int blocks = std::max(1, std::min((n_cfg + threads - 1) / threads, 4 * sm_count(device)));
    if (n_cfg > 0) plan_count_kernel<<<blocks, threads, 0, stream>>>(n_cfg, n_max, order, rb.plan, rb.status, 0);
    plan_prefix_kernel<<<1, 32, 0, stream>>>(cpb, rb.plan);
    if (n_cfg > 0) plan_scatter_kernel<<<blocks, threads, 0, stream>>>(n_cfg, n_max, order, rb.plan, rb.list);
    const int bb = std::max(1, std::min((max_batches + threads - 1) / threads, 4 * sm_count(device)));
    plan_batches_kernel<<<bb, threads, 0, stream>>>(max_batches, cpb, rb.plan, rb.batches);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "planner launch");
    return COS_OK;
}

template <typename T>
static cos_status launch_dp_raw_t(const RawBuffers &rb, const DpLaunch &L, cudaStream_t stream) {
    const Tuning tu = get_tuning(L.n_max, L.precision, L.n_mat);
    const size_t msm = (size_t)L.n_max * L.n_max * kLanes;
    const size_t smem = ((msm * sizeof(T) + 15) & ~size_t(15)) + msm * sizeof(typename CloseOf<T>::type);
    const int threads = tu.warps * 32;
    auto kern = kernel_for_launch<T>(L, threads);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "dp smem attribute");
    DpArgs a;
    memset(&a, 0, sizeof a);
    a.tabs = rb.tabs;
    a.batches = rb.batches;
    a.n_batches = rb.plan + 64;
    a.batch_list = rb.list;
    a.queue = rb.queue;
    a.M = L.M;
    a.moff = L.moff;
    a.mstride = L.mstride;
    a.nf_lanes = L.n_mat;
    a.loop_weight = (double)L.loop_weight;
    for (int l = 0; l < COS_MAX_FLAVORS; ++l) a.sigma[l] = L.sigma[l];
    a.shifts = L.shifts ? 1 : 0;
    a.absmode = L.absmode ? 1 : 0;
    a.scratch = rb.scratch;
    a.slot_elems = (size_t)host_order(L.n_max).max_slots * kLanes;
    a.nslots = dp_slots(L);
    a.smem_n = L.n_max;
    a.prefetch = tu.prefetch;
    a.csub = L.csub;
    a.csub_key = L.csub_key;
    a.out = L.out;
    a.status = rb.status;
    e = cudaMemsetAsync(rb.queue, 0, sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e, "queue reset");
    kern<<<rb.grid, threads, smem, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "dp launch");
    return COS_OK;
}

cos_status launch_dp_raw(const RawBuffers &rb, const DpLaunch &L, cudaStream_t stream) {
    if (L.precision == COS_MIXED) return launch_dp_raw_t<float>(rb, L, stream);
    if (L.precision == COS_DF64) return launch_dp_raw_t<df64>(rb, L, stream);
    return launch_dp_raw_t<double>(rb, L, stream);
}

int dp_max_active_ctas(int precision, int threads, size_t smem) {
    int nb = 0;
    cudaError_t e;
    if (precision == COS_MIXED || precision == COS_DF64) {
        return pair_max_active_ctas(precision, threads, smem);   // these precisions launch the pair kernels
    } else {
        auto k = forward_kernel_for<double, false>(threads);
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, smem);
    }
    return e == cudaSuccess ? nb : 0;
}

bool dp_uses_pair(const DpLaunch &L) {
    return (L.precision == COS_MIXED || L.precision == COS_DF64) && L.csub == nullptr;
}

int dp_configs_per_batch(const DpLaunch &L) {
    return dp_uses_pair(L) ? pair_width(L.precision) * (kLanes / L.n_mat) : kLanes / L.n_mat;
}

size_t dp_smem_bytes(int precision, int n_max) {
    const size_t msm = (size_t)n_max * n_max * kLanes;
    if (precision == COS_MIXED || precision == COS_DF64) return pair_smem_bytes(precision, n_max);
    return msm * 8 + msm * 8;   // double or df64 extension and close matrices
}

cos_status launch_dp(Workspace *ws, const DpLaunch &L, cudaStream_t stream) {
    if (dp_uses_pair(L)) return launch_dp_pair(ws, L, stream);
    if (L.precision == COS_MIXED) return launch_dp_t<float>(ws, L, stream);
    if (L.precision == COS_DF64) return launch_dp_t<df64>(ws, L, stream);
    return launch_dp_t<double>(ws, L, stream);
}

}  // namespace cosdp
