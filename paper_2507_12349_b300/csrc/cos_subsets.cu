// All-subsets mode: the connected sum c(S) of every vertex subset S of each configuration, and
// optionally the full sum a(S) over all (connected or not) decorated covers of S; square and
// bipartite lattices, cycle factors or determinant weights.
//
// Connected sums.  The merged DP rooted at vertex 0 reaches, for every S containing 0, the
// interaction mask mu = 2 * 1_S with no half-visited vertex left: its close is the sum over the
// connected covers of S, up to the global factor 2^(|S|-1) of the untouched-vertex entries.
// The forward kernel stores it when given an output key.  A subset S with smallest vertex m > 0
// only contains vertices >= m, so c(S) comes from the same DP rooted at m on the trailing
// principal submatrices M^l[m.., m..].  One DP launch runs every root of every configuration
// as derived problems of order n_c - m; each derived problem writes its c(S') at
// csub[c * 2^n_max + (S' << m)].
//
// Full sums.  Splitting a cover of S into its connected components, the one that holds min S
// is a connected cover of some T containing min S, and the rest covers S \ T (Methods A, the
// subset recursion relating a and c):
//     a(S) = sum_{T subset of S, min S in T} c(T) a(S \ T),     a(empty) = 1.
// The subset-exponential kernel evaluates it in FP64, one CTA per configuration, subsets
// grouped by size so that each group reads only values of the previous groups.
#include <algorithm>
#include <cmath>
#include <string>

#include "cos_internal.h"

namespace cosdp {

namespace {

int sm_count_of(int device) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    return v > 0 ? v : 1;
}

// Matrix slot of root m inside a configuration's block: roots are stored largest first,
// root m gets room for n_mat (n_max - m)^2 entries.
__host__ __device__ inline int64_t root_offset(int n_max, int n_mat, int m) {
    int64_t off = 0;
    for (int k = n_max; k > n_max - m; --k) off += (int64_t)k * k;
    return off * n_mat;
}

// Derived problem d = c * n_max + m (warp per problem): order n_c - m (0 = empty slot when
// m >= n_c), the trailing principal submatrices of every flavor, and the output key.
__global__ void subset_roots_kernel(int n_cfg, int n_max, int n_mat, const int32_t *order, const int64_t *moff,
                                    const double *M, int32_t *sub_order, int64_t *sub_moff, int64_t *sub_key,
                                    double *sub_M) {
    const int lane = threadIdx.x & 31;
    const int64_t nd = (int64_t)n_cfg * n_max;
    const int64_t blk = root_offset(n_max, n_mat, n_max);
    for (int64_t d = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; d < nd;
         d += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t c = d / n_max;
        const int m = (int)(d % n_max);
        const int nc = order[c];
        const bool valid = nc >= 1 && nc <= n_max;
        const int nd_ord = (valid && m < nc) ? nc - m : 0;
        const int64_t dst = c * blk + root_offset(n_max, n_mat, m);
        if (lane == 0) {
            // an order outside [1, n_max]: -1 at root 0, which the planner flags
            sub_order[d] = valid ? nd_ord : (m == 0 ? -1 : 0);
            sub_moff[d] = dst;
            sub_key[d] = (((c << n_max)) << 4) | m;
        }
        if (nd_ord == 0) continue;
        const double *src = M + moff[c];
        const int per = nd_ord * nd_ord;
        for (int e = lane; e < n_mat * per; e += 32) {
            const int l = e / per, r = e % per;
            const int v = r / nd_ord, j = r % nd_ord;
            sub_M[dst + e] = src[(int64_t)l * nc * nc + (int64_t)(v + m) * nc + (j + m)];
        }
    }
}

// Bipartite layout: per flavor [2 n_c][2 n_c] with index (i * 2 + s); root m keeps rows and
// columns 2m.. (vertices m.., both sublattices).  Derived problem d = c * n_max + m as above.
__global__ void bip_subset_roots_kernel(int n_cfg, int n_max, int n_mat, const int32_t *order, const int64_t *moff,
                                        const double *M4, int32_t *sub_order, int64_t *sub_moff, int64_t *sub_key,
                                        double *sub_M) {
    const int lane = threadIdx.x & 31;
    const int64_t nd = (int64_t)n_cfg * n_max;
    const int64_t blk = 4 * root_offset(n_max, n_mat, n_max);
    for (int64_t d = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; d < nd;
         d += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t c = d / n_max;
        const int m = (int)(d % n_max);
        const int nc = order[c];
        const bool valid = nc >= 1 && nc <= n_max;
        const int nd_ord = (valid && m < nc) ? nc - m : 0;
        const int64_t dst = c * blk + 4 * root_offset(n_max, n_mat, m);
        if (lane == 0) {
            sub_order[d] = valid ? nd_ord : (m == 0 ? -1 : 0);
            sub_moff[d] = dst;
            sub_key[d] = (((c << n_max)) << 4) | m;
        }
        if (nd_ord == 0) continue;
        const double *src = M4 + moff[c];
        const int w = 2 * nd_ord, wc = 2 * nc;
        const int per = w * w;
        for (int e = lane; e < n_mat * per; e += 32) {
            const int l = e / per, r = e % per;
            const int row = r / w, col = r % w;
            sub_M[dst + e] = src[(int64_t)l * wc * wc + (int64_t)(row + 2 * m) * wc + (col + 2 * m)];
        }
    }
}

// Root-0-only keys: the DP runs on the configurations themselves.
__global__ void subset_keys_kernel(int n_cfg, int n_max, int64_t *sub_key) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n_cfg; c += (int64_t)gridDim.x * blockDim.x)
        sub_key[c] = (c << n_max) << 4;
}

// c(S) before the DP: 0 for the empty set and for sets with vertices beyond the configuration's
// order, NaN elsewhere (overwritten by the DP; left NaN for S without vertex 0 in root-0 mode).
__global__ void subset_prefill_kernel(int n_cfg, int n_max, const int32_t *order, double *c_out) {
    const int64_t per = (int64_t)1 << n_max;
    const int64_t total = (int64_t)n_cfg * per;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i >> n_max;
        const uint32_t S = (uint32_t)(i & (per - 1));
        const int nc = min(max(order[c], 0), n_max);
        c_out[i] = (S == 0u || (S >> nc) != 0u) ? 0.0 : __longlong_as_double(0x7ff8000000000000LL);
    }
}

// a(S) for every S of each configuration from its c(T) (one CTA per configuration, grid-stride).
// Shared memory: c and a of one configuration, 2 * 2^n_max doubles.
__global__ void subset_exp_kernel(int n_cfg, int n_max, const int32_t *order, const double *c_in, double *a_out) {
    extern __shared__ double sh[];
    const int per = 1 << n_max;
    double *cs = sh;
    double *as = sh + per;
    for (int c = blockIdx.x; c < n_cfg; c += gridDim.x) {
        __syncthreads();  // the previous configuration's values are no longer read
        const int nc = min(max(order[c], 0), n_max);
        const int pc = 1 << nc;
        const double *cg = c_in + ((int64_t)c << n_max);
        for (int S = threadIdx.x; S < pc; S += blockDim.x) {
            cs[S] = cg[S];
            as[S] = 1.0;  // a(empty); the others are written by their size group below
        }
        __syncthreads();
        for (int k = 1; k <= nc; ++k) {
            for (int S = threadIdx.x; S < pc; S += blockDim.x) {
                if (__popc(S) != k) continue;
                const int low = S & -S;
                const int rest = S ^ low;
                double acc = 0.0;
                // T = low | R for every R subset of rest (R = rest gives c(S) a(empty))
                for (int R = rest;; R = (R - 1) & rest) {
                    const int T = low | R;
                    acc = fma(cs[T], as[S ^ T], acc);
                    if (R == 0) break;
                }
                as[S] = acc;
            }
            __syncthreads();
        }
        double *ag = a_out + ((int64_t)c << n_max);
        for (int S = threadIdx.x; S < per; S += blockDim.x) ag[S] = S < pc ? as[S] : 0.0;
    }
}

}  // namespace

// clow: determinant weights (two spin blocks, loop weight 1, h_sigma = the diagonal shifts);
// the closes of the Alg. 1 sweep are the connected sums themselves (no 2^(|S|-1)).
static cos_status subsets_body(const char *fn, int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                        int n_mat, int loop_weight, const double *h_sigma, const double *d_M,
                        cos_precision precision, int all_roots, double *d_c, double *d_a, bool clow,
                        cudaStream_t s) {
    cos_status st = check_matrices(n_cfg, n_max, d_order, d_moff, n_mat, loop_weight, d_M, precision, d_c, fn);
    if (st != COS_OK) return st;
    if (clow && precision != COS_FP64) {
        set_error(std::string(fn) + ": determinant-weight subsets run in COS_FP64");
        return COS_ERR_UNIMPLEMENTED;
    }
    if (all_roots != 0 && all_roots != 1) {
        set_error(std::string(fn) + ": all_roots must be 0 or 1");
        return COS_ERR_ARG;
    }
    if (d_a && !all_roots) {
        set_error(std::string(fn) + ": the full sums a(S) need every root (all_roots = 1)");
        return COS_ERR_ARG;
    }
    if (n_cfg == 0) return COS_OK;
    if (all_roots && (int64_t)n_cfg * n_max > (int64_t)INT32_MAX) {
        set_error(std::string(fn) + ": n_cfg * n_max exceeds the derived-problem limit 2^31 - 1");
        return COS_ERR_ARG;
    }
    std::string err;
    Workspace *ws = get_workspace(s, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    const int nsm = sm_count_of(ws->device);
    const int threads = 256;
    const int64_t total = (int64_t)n_cfg << n_max;
    const int pf_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + threads - 1) / threads, 8LL * nsm));
    subset_prefill_kernel<<<pf_blocks, threads, 0, s>>>(n_cfg, n_max, d_order, d_c);

    DpLaunch L;
    L.n_max = n_max;
    L.n_mat = n_mat;
    L.loop_weight = loop_weight;
    for (int l = 0; l < n_mat; ++l) {
        L.sigma[l] = h_sigma ? h_sigma[l] : 0.0;
        if (L.sigma[l] != 0.0 && !clow) L.shifts = true;
    }
    L.clow = clow;
    L.precision = precision;
    L.csub = d_c;
    if (all_roots) {
        const size_t nd = (size_t)n_cfg * n_max;
        const size_t mdoubles = (size_t)n_cfg * (size_t)root_offset(n_max, n_mat, n_max);
        st = ensure((void **)&ws->sub_order, &ws->sub_cap, nd, sizeof(int32_t), "subset orders");
        if (st == COS_OK) st = ensure((void **)&ws->sub_moff, &ws->sub_moff_cap, nd, sizeof(int64_t), "subset offsets");
        if (st == COS_OK) st = ensure((void **)&ws->sub_key, &ws->sub_key_cap, nd, sizeof(int64_t), "subset keys");
        if (st == COS_OK) st = ensure((void **)&ws->sub_M, &ws->sub_M_cap, mdoubles, sizeof(double), "subset matrices");
        if (st != COS_OK) return st;
        const int rb = (int)std::max<size_t>(1, std::min<size_t>((nd * 32 + threads - 1) / threads, 8 * (size_t)nsm));
        subset_roots_kernel<<<rb, threads, 0, s>>>(n_cfg, n_max, n_mat, d_order, d_moff, d_M, ws->sub_order,
                                                   ws->sub_moff, ws->sub_key, ws->sub_M);
        L.n_cfg = (int)nd;
        L.order = ws->sub_order;
        L.M = ws->sub_M;
        L.moff = ws->sub_moff;
        L.csub_key = ws->sub_key;
        L.allow_empty = true;
    } else {
        st = ensure((void **)&ws->sub_key, &ws->sub_key_cap, (size_t)n_cfg, sizeof(int64_t), "subset keys");
        if (st != COS_OK) return st;
        const int kb = std::max(1, std::min((n_cfg + threads - 1) / threads, 8 * nsm));
        subset_keys_kernel<<<kb, threads, 0, s>>>(n_cfg, n_max, ws->sub_key);
        L.n_cfg = n_cfg;
        L.order = d_order;
        L.M = d_M;
        L.moff = d_moff;
        L.csub_key = ws->sub_key;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "subset set-up launch");
    st = run_dp(ws, L, nullptr, s);
    if (st != COS_OK || !d_a) return st;
    const size_t smem = ((size_t)2 << n_max) * sizeof(double);  // c and a of one configuration
    e = cudaFuncSetAttribute(subset_exp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "subset exponential smem attribute");
    const int eb = std::max(1, std::min(n_cfg, 16 * nsm));
    subset_exp_kernel<<<eb, threads, smem, s>>>(n_cfg, n_max, d_order, d_c, d_a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "subset exponential launch");
    return COS_OK;
}

// Bipartite lattices: the same mode on the sublattice-resolved sweep (FP64).  Orders up to
// COS_BIP_NMAX; h_sigma2 [n_mat][2] (cycle factors) or the [2][2] diagonal shifts (clow).
static cos_status bip_subsets_body(const char *fn, int n_cfg, int n_max, const int32_t *d_order,
                                   const int64_t *d_moff, int n_mat, int loop_weight, const double *h_sigma2,
                                   const double *d_M4, cos_precision precision, int all_roots, double *d_c,
                                   double *d_a, bool clow, cudaStream_t s) {
    if (n_cfg < 0 || n_mat < 1 || n_mat > COS_MAX_FLAVORS || loop_weight < 1) {
        set_error(std::string(fn) + ": n_cfg < 0, n_mat outside [1, 8] or loop_weight < 1");
        return COS_ERR_ARG;
    }
    if (n_max < 1 || n_max > COS_BIP_NMAX) {
        set_error(std::string(fn) + ": n_max outside [1, 9]");
        return COS_ERR_ORDER;
    }
    if (precision != COS_FP64) {
        set_error(std::string(fn) + ": the bipartite all-subsets mode runs in COS_FP64");
        return precision == COS_MIXED || precision == COS_DF64 ? COS_ERR_UNIMPLEMENTED : COS_ERR_ARG;
    }
    if (all_roots != 0 && all_roots != 1) {
        set_error(std::string(fn) + ": all_roots must be 0 or 1");
        return COS_ERR_ARG;
    }
    if (d_a && !all_roots) {
        set_error(std::string(fn) + ": the full sums a(S) need every root (all_roots = 1)");
        return COS_ERR_ARG;
    }
    if (n_cfg > 0 && (!d_order || !d_moff || !d_M4 || !d_c)) {
        set_error(std::string(fn) + ": null device pointer");
        return COS_ERR_ARG;
    }
    if (n_cfg == 0) return COS_OK;
    if (all_roots && (int64_t)n_cfg * n_max > (int64_t)INT32_MAX) {
        set_error(std::string(fn) + ": n_cfg * n_max exceeds the derived-problem limit 2^31 - 1");
        return COS_ERR_ARG;
    }
    std::string err;
    Workspace *ws = get_workspace(s, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    const int nsm = sm_count_of(ws->device);
    const int threads = 256;
    const int64_t total = (int64_t)n_cfg << n_max;
    const int pf_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + threads - 1) / threads, 8LL * nsm));
    subset_prefill_kernel<<<pf_blocks, threads, 0, s>>>(n_cfg, n_max, d_order, d_c);
    cos_status st;
    if (all_roots) {
        const size_t nd = (size_t)n_cfg * n_max;
        const size_t mdoubles = (size_t)n_cfg * (size_t)(4 * root_offset(n_max, n_mat, n_max));
        st = ensure((void **)&ws->sub_order, &ws->sub_cap, nd, sizeof(int32_t), "subset orders");
        if (st == COS_OK) st = ensure((void **)&ws->sub_moff, &ws->sub_moff_cap, nd, sizeof(int64_t), "subset offsets");
        if (st == COS_OK) st = ensure((void **)&ws->sub_key, &ws->sub_key_cap, nd, sizeof(int64_t), "subset keys");
        if (st == COS_OK) st = ensure((void **)&ws->sub_M, &ws->sub_M_cap, mdoubles, sizeof(double), "subset matrices");
        if (st != COS_OK) return st;
        const int rb = (int)std::max<size_t>(1, std::min<size_t>((nd * 32 + threads - 1) / threads, 8 * (size_t)nsm));
        bip_subset_roots_kernel<<<rb, threads, 0, s>>>(n_cfg, n_max, n_mat, d_order, d_moff, d_M4, ws->sub_order,
                                                       ws->sub_moff, ws->sub_key, ws->sub_M);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "bipartite subset set-up launch");
        st = bip_subsets_dp(ws, (int)nd, n_max, ws->sub_order, ws->sub_moff, n_mat, loop_weight, h_sigma2, ws->sub_M,
                            clow, d_c, ws->sub_key, true, s);
    } else {
        st = ensure((void **)&ws->sub_key, &ws->sub_key_cap, (size_t)n_cfg, sizeof(int64_t), "subset keys");
        if (st != COS_OK) return st;
        const int kb = std::max(1, std::min((n_cfg + threads - 1) / threads, 8 * nsm));
        subset_keys_kernel<<<kb, threads, 0, s>>>(n_cfg, n_max, ws->sub_key);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "bipartite subset set-up launch");
        st = bip_subsets_dp(ws, n_cfg, n_max, d_order, d_moff, n_mat, loop_weight, h_sigma2, d_M4, clow, d_c,
                            ws->sub_key, false, s);
    }
    if (st != COS_OK || !d_a) return st;
    const size_t smem = ((size_t)2 << n_max) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(subset_exp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "subset exponential smem attribute");
    const int eb = std::max(1, std::min(n_cfg, 16 * nsm));
    subset_exp_kernel<<<eb, threads, smem, s>>>(n_cfg, n_max, d_order, d_c, d_a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "subset exponential launch");
    return COS_OK;
}

}  // namespace cosdp

using namespace cosdp;

COS_INTERNAL_API cos_status cos_connected_sum_bipartite_subsets(int n_cfg, int n_max, const int32_t *d_order,
                                                          const int64_t *d_moff, int n_mat, int loop_weight,
                                                          const double *h_sigma2, const double *d_M4,
                                                          cos_precision precision, int all_roots, double *d_c,
                                                          double *d_a, cos_stream_t stream) {
    return bip_subsets_body("cos_connected_sum_bipartite_subsets", n_cfg, n_max, d_order, d_moff, n_mat, loop_weight,
                            h_sigma2, d_M4, precision, all_roots, d_c, d_a, false, (cudaStream_t)stream);
}

COS_INTERNAL_API cos_status cos_connected_det_bipartite_subsets(int n_cfg, int n_max, const int32_t *d_order,
                                                          const int64_t *d_moff, const double *h_alpha2,
                                                          const double *d_M4, cos_precision precision, int all_roots,
                                                          double *d_c, double *d_a, cos_stream_t stream) {
    return bip_subsets_body("cos_connected_det_bipartite_subsets", n_cfg, n_max, d_order, d_moff, 2, 1, h_alpha2,
                            d_M4, precision, all_roots, d_c, d_a, true, (cudaStream_t)stream);
}

COS_INTERNAL_API cos_status cos_connected_sum_subsets(int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                                                int n_mat, int loop_weight, const double *h_sigma,
                                                const double *d_M, cos_precision precision, int all_roots,
                                                double *d_c, double *d_a, cos_stream_t stream) {
    return subsets_body("cos_connected_sum_subsets", n_cfg, n_max, d_order, d_moff, n_mat, loop_weight, h_sigma, d_M,
                        precision, all_roots, d_c, d_a, false, (cudaStream_t)stream);
}

COS_INTERNAL_API cos_status cos_connected_det_subsets(int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                                                const double *h_alpha, const double *d_M, cos_precision precision,
                                                int all_roots, double *d_c, double *d_a, cos_stream_t stream) {
    return subsets_body("cos_connected_det_subsets", n_cfg, n_max, d_order, d_moff, 2, 1, h_alpha, d_M, precision,
                        all_roots, d_c, d_a, true, (cudaStream_t)stream);
}
