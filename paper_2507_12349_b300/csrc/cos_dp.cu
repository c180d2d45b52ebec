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
//     global ring of 2 (3 with shift parameters) layer slots laid out [slot][lane].
//
// Recurrence (push form, per row = mask mu, head h, lane flavor l, endpoints v in Vrow):
//   close   csum(mu)            += sum_v O(mu,h,v) M[v][h]                      (Alg. 2 Close)
//   extend  O(mu+e_j, h, j)     (+)= d_j = sum_v O(mu,h,v) M[v][j], mu_j <= 1     (Alg. 2 Extend)
//   shift   O(mu+2e_j, h, j)     = -sigma_l d_j,  mu_j = 0                     (Alg. 3 shift head)
//   after all rows of mu:  C(mu) = -w sum_{lanes of the configuration} csum   (flavor sum)
//            mu has a 1 -> O(mu+e_k, k, k) = C(mu) in every flavor, k = min{i: mu_i = 1}
//            mu full    -> c = 2^(n-1) C(mu)
// The factor 2 for entering an untouched vertex (either of its two points) is the same on
// every path -- each vertex other than 0 is entered from mu_j = 0 exactly once -- so it is
// pulled out as the global 2^(n-1); the start with a shifted vertex 0 keeps its 2 (-2 sigma).
// Each target slot receives one plain store before any read-modify-write (see the cases in
// process_mask), so slots never need clearing between batches.
#include <algorithm>
#include <cstring>

#include "cos_internal.h"

namespace cosdp {

__constant__ uint32_t c_p3[COS_NMAX + 2] = {1u, 3u, 9u, 27u, 81u, 243u, 729u, 2187u, 6561u,
                                           19683u, 59049u, 177147u, 531441u, 1594323u};

struct DpArgs {
    const OrderTab *tabs;       // [COS_NMAX + 1]
    const int4 *batches;        // {n, start, count, 0}
    const int *n_batches;
    const int *batch_list;
    int *queue;
    const double *M;
    const int64_t *moff;
    int64_t mstride;
    int nf_lanes;
    double loop_weight;
    double sigma[COS_MAX_FLAVORS];
    int shifts;
    int absmode;
    void *scratch;
    size_t slot_elems;          // elements per layer slot (max layer slots * 32)
    int nslots;
    int smem_n;                 // order used for the shared-memory layout stride (n_max)
    double *out;
    int *status;
};

template <typename T>
struct Prec;
template <>
struct Prec<double> {
    static __device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
};
template <>
struct Prec<float> {
    static __device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
};

// One row (mu, h): load its NV endpoint states, accumulate the close, push every extension.
template <typename T, int NV>
__device__ __forceinline__ void do_row(const T *__restrict__ src, T *__restrict__ dst1, T *__restrict__ dst2,
                                       const T *__restrict__ Ms, const double *__restrict__ Md,
                                       const uint32_t *__restrict__ rank3, uint32_t Vrow, uint32_t A, uint32_t B,
                                       uint32_t J, uint32_t code, uint32_t off, int h, int hidx, int nA, int n,
                                       bool needclose, bool shifts, T negsig, int lane, double &csum) {
    T o[NV];
    int vs[NV];
    const T *row = src + (size_t)(off + (uint32_t)(hidx * nA)) * kLanes + lane;
    uint32_t vv = Vrow;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        const int v = __ffs(vv) - 1;
        vv &= vv - 1u;
        o[t] = row[__popc(A & ((1u << v) - 1u)) * kLanes];
        vs[t] = v * n * kLanes + lane;
    }
    if (needclose) {
#pragma unroll
        for (int t = 0; t < NV; ++t) csum = fma((double)o[t], Md[vs[t] + h * kLanes], csum);
    }
    const uint32_t hlow = (1u << h) - 1u;
    for (uint32_t jj = J; jj; jj &= jj - 1u) {
        const int j = __ffs(jj) - 1;
        T d = T(0);
#pragma unroll
        for (int t = 0; t < NV; ++t) d = Prec<T>::fma_(o[t], Ms[vs[t] + j * kLanes], d);
        const uint32_t bj = 1u << j;
        const bool untouched = !(A & bj);
        const uint32_t A1 = A | bj;
        const uint32_t B1 = untouched ? B : (B | bj);
        const int nA1 = __popc(A1);
        const int ai1 = __popc(A1 & (bj - 1u));
        const int hi1 = __popc(head_set(B1, A1 & ~B1) & hlow);
        const uint32_t off1 = __ldg(rank3 + code + c_p3[j]);
        T *tp = dst1 + (size_t)(off1 + (uint32_t)(hi1 * nA1 + ai1)) * kLanes + lane;
        if (untouched) {
            // mu_j = 0 -> 1: the only writer of this slot.
            *tp = d;
            if (shifts) {
                // mu_j = 0 -> 2 through a shift point: first (plain) writer of the slot; the
                // extension from mu+e_j adds to it one layer later.
                const uint32_t B2 = B | bj;
                const int hi2 = __popc(head_set(B2, A1 & ~B2) & hlow);
                const uint32_t off2 = __ldg(rank3 + code + 2u * c_p3[j]);
                dst2[(size_t)(off2 + (uint32_t)(hi2 * nA1 + ai1)) * kLanes + lane] = negsig * d;
            }
        } else if (shifts && j != 0) {
            *tp += d;
        } else {
            // mu_j = 1 -> 2 without shift sources (j = 0: the seed of the new head at vertex 0,
            // issued later by this same thread, adds to it).
            *tp = d;
        }
    }
}

template <typename T>
__device__ __forceinline__ void row_dispatch(int nv, const T *src, T *dst1, T *dst2, const T *Ms, const double *Md,
                                             const uint32_t *rank3, uint32_t Vrow, uint32_t A, uint32_t B, uint32_t J,
                                             uint32_t code, uint32_t off, int h, int hidx, int nA, int n,
                                             bool needclose, bool shifts, T negsig, int lane, double &csum) {
#define COS_ROW(K)                                                                                          \
    case K:                                                                                                 \
        do_row<T, K>(src, dst1, dst2, Ms, Md, rank3, Vrow, A, B, J, code, off, h, hidx, nA, n, needclose,   \
                     shifts, negsig, lane, csum);                                                           \
        break;
    switch (nv) {
        COS_ROW(1)
        COS_ROW(2)
        COS_ROW(3)
        COS_ROW(4)
        COS_ROW(5)
        COS_ROW(6)
        COS_ROW(7)
        COS_ROW(8)
        COS_ROW(9)
        COS_ROW(10)
        COS_ROW(11)
        COS_ROW(12)
        default:
            break;
    }
#undef COS_ROW
}

template <typename T>
__global__ void __launch_bounds__(512) dp_forward_kernel(const __grid_constant__ DpArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_batch;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int nsm = a.smem_n * a.smem_n * kLanes;
    T *Ms = reinterpret_cast<T *>(smem_raw);
    const double *Md = sizeof(T) == sizeof(double)
                           ? reinterpret_cast<const double *>(smem_raw)
                           : reinterpret_cast<const double *>(smem_raw + ((nsm * sizeof(T) + 15) & ~size_t(15)));
    double *Mdw = const_cast<double *>(Md);
    T *ring = reinterpret_cast<T *>(a.scratch) + (size_t)blockIdx.x * a.nslots * a.slot_elems;
    const int nfl = a.nf_lanes;
    const int lam = lane % nfl;
    const int ci = lane / nfl;
    const double sgn = a.absmode ? 1.0 : -1.0;
    const double sig = a.absmode ? fabs(a.sigma[lam]) : a.sigma[lam];
    const bool shifts = a.shifts != 0;
    const int nbatch = *a.n_batches;

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
        // Matrices of the batch -> shared memory [v][j][lane].
        for (int e = warp; e < n * n; e += nwarps) {
            double val = active ? Mc[e] : 0.0;
            if (a.absmode) val = fabs(val);
            Ms[e * kLanes + lane] = (T)val;
            if (sizeof(T) != sizeof(double)) Mdw[e * kLanes + lane] = val;
        }
        // Start: the loop through the normal point of vertex 0 (layer 1, mask e_0, slot 0).
        if (warp == 0) ring[(1 % a.nslots) * a.slot_elems + lane] = T(1);
        __syncthreads();

        const uint32_t full = (1u << n) - 1u;
        const T negsig = (T)(sgn * sig);
        for (int ell = 1; ell <= 2 * n; ++ell) {
            const T *src = ring + (size_t)(ell % a.nslots) * a.slot_elems;
            T *dst1 = ring + (size_t)((ell + 1) % a.nslots) * a.slot_elems;
            T *dst2 = ring + (size_t)((ell + 2) % a.nslots) * a.slot_elems;
            const uint32_t first = tab.layer_first[ell];
            const uint32_t cnt = tab.layer_count[ell];
            for (uint32_t mi = warp; mi < cnt; mi += nwarps) {
                const uint4 mk = __ldg(reinterpret_cast<const uint4 *>(tab.masks + first + mi));
                const uint32_t A = mk.x & 0xFFFFu, B = mk.x >> 16, code = mk.y, off = mk.z;
                const uint32_t ones = A & ~B;
                const uint32_t H = head_set(B, ones);
                const uint32_t J = full & ~B;
                const int nA = __popc(A);
                const bool needclose = (ones != 0u) || (B == full);
                double csum = 0.0;
                for (uint32_t hh = H; hh; hh &= hh - 1u) {
                    const int h = __ffs(hh) - 1;
                    const int hidx = __popc(H & ((1u << h) - 1u));
                    const uint32_t Vrow = row_vmask(A, ones, h);
                    row_dispatch<T>(__popc(Vrow), src, dst1, dst2, Ms, Md, tab.rank3, Vrow, A, B, J, code, off, h,
                                    hidx, nA, n, needclose, shifts, negsig, lane, csum);
                }
                if (!needclose) continue;  // no half-visited vertex and not full: disconnected, dropped
                // Flavor sum of the loop-closing weight over the lanes of this configuration.
                double tot = csum;
                if (nfl > 1) {
                    const int base = ci * nfl;
                    tot = 0.0;
                    for (int g = 0; g < nfl; ++g) tot += __shfl_sync(0xFFFFFFFFu, csum, (base + g) & 31);
                }
                const double C = sgn * a.loop_weight * tot;
                if (ones) {
                    const int k = __ffs(ones) - 1;
                    const uint32_t bk = 1u << k;
                    const uint32_t B1 = B | bk;
                    const int hi1 = __popc(head_set(B1, A & ~B1) & (bk - 1u));
                    const int ai1 = __popc(A & (bk - 1u));
                    const uint32_t off1 = __ldg(tab.rank3 + code + c_p3[k]);
                    T *tp = dst1 + (size_t)(off1 + (uint32_t)(hi1 * nA + ai1)) * kLanes + lane;
                    double val = C;
                    if (ell == 1 && shifts) val += sgn * 2.0 * sig;  // vertex 0 carries a shift point
                    if (k == 0) *tp += (T)val;                        // the extension into 0' wrote it
                    else *tp = (T)val;
                } else if (active && lam == 0) {
                    const double c = ldexp(C, n - 1);
                    a.out[cfg] = c;
                    if (!isfinite(c)) atomicOr(a.status, kStatusNonFinite);
                }
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------ batch planner
// Sorts configurations by order (largest first) into batches of `cpb` configurations.
// plan layout: [0,16) counts, [16,32) cursors, [32,48) bucket starts, [48,64) batch starts, [64] n_batches

__global__ void plan_count_kernel(int n_cfg, int n_max, const int32_t *order, int *plan, int *status) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cfg; c += gridDim.x * blockDim.x) {
        const int n = order[c];
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
                               cudaStream_t stream) {
    const int max_batches = (n_cfg + cpb - 1) / cpb + COS_NMAX;
    cos_status st = ensure((void **)&ws->batch_list, &ws->batch_cap, (size_t)n_cfg + 1, sizeof(int), "batch list");
    if (st != COS_OK) return st;
    st = ensure((void **)&ws->batches, &ws->batches_cap, (size_t)max_batches, sizeof(int4), "batch table");
    if (st != COS_OK) return st;
    cudaError_t e = cudaMemsetAsync(ws->plan_counts, 0, 80 * sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e, "planner memset");
    const int threads = 256;
    const int blocks = std::max(1, std::min((n_cfg + threads - 1) / threads, 4 * sm_count(ws->device)));
    if (n_cfg > 0) plan_count_kernel<<<blocks, threads, 0, stream>>>(n_cfg, n_max, order, ws->plan_counts, ws->status);
    plan_prefix_kernel<<<1, 32, 0, stream>>>(cpb, ws->plan_counts);
    if (n_cfg > 0) plan_scatter_kernel<<<blocks, threads, 0, stream>>>(n_cfg, n_max, order, ws->plan_counts, ws->batch_list);
    const int bb = std::max(1, std::min((max_batches + threads - 1) / threads, 4 * sm_count(ws->device)));
    plan_batches_kernel<<<bb, threads, 0, stream>>>(max_batches, cpb, ws->plan_counts, ws->batches);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "planner launch");
    return COS_OK;
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
    const int nslots = L.shifts ? 3 : 2;
    const size_t slot_elems = (size_t)host_order(L.n_max).max_slots * kLanes;
    const size_t per_cta = (size_t)nslots * slot_elems * sizeof(T);
    const int cpb = kLanes / nfl;
    const int max_batches = (L.n_cfg + cpb - 1) / cpb + COS_NMAX;
    int grid = std::max(1, std::min(nsm * tu.ctas_per_sm, max_batches));
    // Keep the layer scratch inside the free device memory (leave headroom for the caller).
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
        const size_t avail = ws->scratch_bytes + (size_t)(0.85 * (double)free_b);
        while (grid > 1 && (size_t)grid * per_cta > avail) grid = std::max(1, grid / 2);
    }
    cos_status st = ensure(&ws->scratch, &ws->scratch_bytes, (size_t)grid * per_cta, 1, "layer scratch");
    if (st != COS_OK) return st;
    const int threads = tu.warps * 32;
    const size_t msm = (size_t)L.n_max * L.n_max * kLanes;
    size_t smem = ((msm * sizeof(T) + 15) & ~size_t(15));
    if (sizeof(T) != sizeof(double)) smem += msm * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(dp_forward_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
    a.out = L.out;
    a.status = ws->status;
    e = cudaMemsetAsync(ws->queue, 0, sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e, "queue reset");
    dp_forward_kernel<T><<<grid, threads, smem, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "dp launch");
    return COS_OK;
}

// ------------------------------------------------------------------ raw-buffer launchers

int dp_slots(const DpLaunch &L) { return L.shifts ? 3 : 2; }
size_t dp_state_bytes(const DpLaunch &L) { return L.precision == COS_MIXED ? sizeof(float) : sizeof(double); }

cos_status launch_plan_raw(const RawBuffers &rb, int n_cfg, int n_max, const int32_t *order, int cpb, int device,
                           cudaStream_t stream) {
    const int max_batches = (n_cfg + cpb - 1) / cpb + COS_NMAX;
    cudaError_t e = cudaMemsetAsync(rb.plan, 0, 80 * sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e, "planner memset");
    const int threads = 256;
    const int blocks = std::max(1, std::min((n_cfg + threads - 1) / threads, 4 * sm_count(device)));
    if (n_cfg > 0) plan_count_kernel<<<blocks, threads, 0, stream>>>(n_cfg, n_max, order, rb.plan, rb.status);
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
    size_t smem = ((msm * sizeof(T) + 15) & ~size_t(15));
    if (sizeof(T) != sizeof(double)) smem += msm * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(dp_forward_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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
    a.out = L.out;
    a.status = rb.status;
    e = cudaMemsetAsync(rb.queue, 0, sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e, "queue reset");
    dp_forward_kernel<T><<<rb.grid, tu.warps * 32, smem, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "dp launch");
    return COS_OK;
}

cos_status launch_dp_raw(const RawBuffers &rb, const DpLaunch &L, cudaStream_t stream) {
    if (L.precision == COS_MIXED) return launch_dp_raw_t<float>(rb, L, stream);
    return launch_dp_raw_t<double>(rb, L, stream);
}

cos_status launch_dp(Workspace *ws, const DpLaunch &L, cudaStream_t stream) {
    if (L.precision == COS_MIXED) return launch_dp_t<float>(ws, L, stream);
    return launch_dp_t<double>(ws, L, stream);
}

}  // namespace cosdp
