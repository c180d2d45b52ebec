// K-TAB (propagator tables) and K-GATHER (per-configuration matrices).
//
// Methods A, square lattice: xi_l(k) = -2t [cos k_x + cos k_y] - mu_l + alpha_l with
// k = 2 pi m / L, and G0_l(r, tau) = -(1/L^2) sum_k cos(k.r) exp(-xi tau)(1 - n_F(xi)) for
// 0 < tau < beta (G0 = -<T c c^+>), antiperiodic in tau.  Tables hold tau_m = m beta/(n_tau-1).
#include <cmath>
#include <cstring>

#include "cos_internal.h"

namespace cosdp {

// xi for every (matrix, momentum), momentum index k = m_x + L m_y; cosines via cospi.
__global__ void xi_kernel(int L, int n_mat, double t, const double *mu_minus_alpha, double *xi, double *coslut) {
    const int total = n_mat * L * L;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int l = i / (L * L), k = i % (L * L);
        const int mx = k % L, my = k / L;
        xi[i] = -2.0 * t * (cospi(2.0 * mx / L) + cospi(2.0 * my / L)) - mu_minus_alpha[l];
    }
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < L; q += gridDim.x * blockDim.x)
        coslut[q] = cospi(2.0 * q / L);
}

// w = exp(-xi tau)(1 - n_F(xi)) in the overflow-free form of each sign of xi; with deriv,
// also w (tau - beta n_F) = -dw/dxi = dw/dmu.
__global__ void weight_kernel(int LL, int n_mat, int n_tau, double beta, const double *xi, double *W, double *Wd) {
    const size_t total = (size_t)n_mat * LL * n_tau;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(i % n_tau);
        const size_t lk = i / n_tau;
        const double x = xi[lk];
        const double tau = beta * m / (n_tau - 1);
        double w, nf;
        if (x >= 0.0) {
            const double e = exp(-beta * x);
            w = exp(-x * tau) / (1.0 + e);
            nf = e / (1.0 + e);
        } else {
            const double e = exp(beta * x);
            w = exp(x * (beta - tau)) / (1.0 + e);
            nf = 1.0 / (1.0 + e);
        }
        W[i] = w;
        if (Wd) Wd[i] = w * (tau - beta * nf);
    }
}

// G[l][r][m] = -(1/L^2) sum_k cos(k.r) W[l][k][m]; cos(k.r) = cos(2 pi ((m_x x + m_y y) mod L) / L).
__global__ void ksum_kernel(int L, int n_mat, int n_tau, const double *W, const double *coslut, double *G) {
    extern __shared__ double s_cos[];
    for (int q = threadIdx.x; q < L; q += blockDim.x) s_cos[q] = coslut[q];
    __syncthreads();
    const int LL = L * L;
    const size_t total = (size_t)n_mat * LL * n_tau;
    const double scale = -1.0 / (double)LL;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(i % n_tau);
        const int r = (int)((i / n_tau) % LL);
        const int l = (int)(i / ((size_t)n_tau * LL));
        const int x = r % L, y = r / L;
        const double *Wl = W + (size_t)l * LL * n_tau + m;
        double acc = 0.0;
        for (int my = 0; my < L; ++my) {
            const int qy = (my * y) % L;
            for (int mx = 0; mx < L; ++mx) {
                const int q = (mx * x + qy) % L;
                acc = fma(s_cos[q], Wl[(size_t)(mx + L * my) * n_tau], acc);
            }
        }
        G[i] = scale * acc;
    }
}

// One warp per configuration: lanes walk the n_mat * n * n entries.
__global__ void gather_kernel(const double *__restrict__ G, int L, int n_tau, double beta, int n_mat, int n_cfg,
                              const int32_t *__restrict__ order, const int64_t *__restrict__ offset,
                              const int32_t *__restrict__ site, const double *__restrict__ tau,
                              const int64_t *__restrict__ moff, int64_t mstride, double *__restrict__ M,
                              int *status) {
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int LL = L * L;
    const double scale = (double)(n_tau - 1) / beta;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_cfg; c += warps) {
        const int n = order[c];
        // an order above the stride layout's n_max would spill into the next configuration
        if (n < 1 || n > COS_NMAX || (!moff && (int64_t)n_mat * n * n > mstride)) {
            if (lane == 0) atomicOr(status, kStatusOrder);
            continue;
        }
        const int64_t o = offset[c];
        double *Mc = M + (moff ? moff[c] : (int64_t)c * mstride);
        const int nn = n * n;
        for (int e = lane; e < n_mat * nn; e += 32) {
            const int l = e / nn, i = (e / n) % n, j = e % n;
            const int si = site[o + i], sj = site[o + j];
            if (si < 0 || si >= LL || sj < 0 || sj >= LL) {
                atomicOr(status, kStatusSite);
                Mc[e] = nan("");
                continue;
            }
            const int dx = ((si % L) - (sj % L) + L) % L;
            const int dy = ((si / L) - (sj / L) + L) % L;
            const int r = dx + L * dy;
            const double dt = tau[o + i] - tau[o + j];
            double s = 1.0, tt = dt;
            if (dt <= 0.0) {
                s = -1.0;
                tt = dt + beta;
            }
            const double x = tt * scale;
            int m = (int)floor(x);
            m = max(0, min(m, n_tau - 2));
            const double f = x - m;
            const double *row = G + ((size_t)l * LL + r) * n_tau + m;
            const double g0 = row[0], g1 = row[1];
            Mc[e] = s * fma(f, g1 - g0, g0);
        }
    }
}

cos_status launch_gather(const cos_tables *t, int n_cfg, const int32_t *order, const int64_t *offset,
                         const int32_t *site, const double *tau, const int64_t *moff, int64_t mstride, double *M,
                         int *status, cudaStream_t stream) {
    if (n_cfg == 0) return COS_OK;
    const int threads = 256;
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, t->device);
    const int blocks = std::max(1, std::min((n_cfg * 32 + threads - 1) / threads, 8 * nsm));
    gather_kernel<<<blocks, threads, 0, stream>>>(t->d_G, t->model.L, t->model.n_tau, t->model.beta, t->n_mat, n_cfg,
                                                   order, offset, site, tau, moff, mstride, M, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "gather launch");
    return COS_OK;
}

// Builds G (and dG/dmu when `deriv`) for the distinct flavors of `t`.
static cos_status build_tables(cos_tables *t, bool deriv, cudaStream_t stream) {
    const int L = t->model.L, LL = L * L, n_tau = t->model.n_tau, n_mat = t->n_mat;
    const size_t nW = (size_t)n_mat * LL * n_tau;
    double *d_ma = nullptr, *d_xi = nullptr, *d_cos = nullptr, *d_W = nullptr, *d_Wd = nullptr;
    double h_ma[COS_MAX_FLAVORS];
    for (int l = 0; l < n_mat; ++l) h_ma[l] = t->mu[l] - t->alpha[l];
    cudaError_t e = cudaMalloc(&d_ma, sizeof(double) * n_mat);
    if (e == cudaSuccess) e = cudaMalloc(&d_xi, sizeof(double) * n_mat * LL);
    if (e == cudaSuccess) e = cudaMalloc(&d_cos, sizeof(double) * L);
    if (e == cudaSuccess) e = cudaMalloc(&d_W, sizeof(double) * nW);
    if (e == cudaSuccess && deriv) e = cudaMalloc(&d_Wd, sizeof(double) * nW);
    double **target = deriv ? &t->d_dG : &t->d_G;
    if (e == cudaSuccess && !*target) e = cudaMalloc(target, sizeof(double) * nW);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_ma, h_ma, sizeof(double) * n_mat, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) {
        xi_kernel<<<std::max(1, (n_mat * LL + 255) / 256), 256, 0, stream>>>(L, n_mat, t->model.t, d_ma, d_xi, d_cos);
        const int wb = (int)std::min<size_t>((nW + 255) / 256, 65535);
        weight_kernel<<<wb, 256, 0, stream>>>(LL, n_mat, n_tau, t->model.beta, d_xi, d_W, d_Wd);
        ksum_kernel<<<wb, 256, L * sizeof(double), stream>>>(L, n_mat, n_tau, deriv ? d_Wd : d_W, d_cos, *target);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFree(d_ma);
    cudaFree(d_xi);
    cudaFree(d_cos);
    cudaFree(d_W);
    cudaFree(d_Wd);
    if (e != cudaSuccess) return cuda_fail(e, "propagator tables");
    return COS_OK;
}

cos_status ensure_dtables(cos_tables *t, cudaStream_t stream) {
    if (t->d_dG) return COS_OK;
    return build_tables(t, true, stream);
}

}  // namespace cosdp

extern "C" cos_status cos_build_propagators(const cos_model *m, cos_stream_t stream, cos_tables **out) {
    using namespace cosdp;
    if (!m || !out) {
        set_error("cos_build_propagators: null argument");
        return COS_ERR_ARG;
    }
    *out = nullptr;
    if (m->L < 1 || m->L > 256 || m->n_tau < 2 || m->n_tau > 65536 || m->n_flavors < 1 ||
        m->n_flavors > COS_MAX_FLAVORS || !(m->beta > 0.0) || m->U == 0.0 || !m->mu || !m->alpha) {
        set_error("cos_build_propagators: model out of range");
        return COS_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cos_tables *t = new cos_tables();
    t->device = dev;
    t->mu.assign(m->mu, m->mu + m->n_flavors);
    t->alpha.assign(m->alpha, m->alpha + m->n_flavors);
    t->model = *m;
    t->model.mu = t->mu.data();
    t->model.alpha = t->alpha.data();
    bool sym = true;
    for (int l = 1; l < m->n_flavors; ++l)
        if (t->mu[l] != t->mu[0] || t->alpha[l] != t->alpha[0]) sym = false;
    t->symmetric = sym ? 1 : 0;
    t->n_mat = sym ? 1 : m->n_flavors;
    for (int l = 0; l < COS_MAX_FLAVORS; ++l) t->sigma[l] = l < m->n_flavors ? t->alpha[l] / m->U : 0.0;
    t->d_G = nullptr;
    t->d_dG = nullptr;
    cos_status st = build_tables(t, false, (cudaStream_t)stream);
    if (st != COS_OK) {
        cudaFree(t->d_G);
        delete t;
        return st;
    }
    *out = t;
    return COS_OK;
}

extern "C" cos_status cos_free_tables(cos_tables *t) {
    if (!t) return COS_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(t->device);
    cudaFree(t->d_G);
    cudaFree(t->d_dG);
    cudaSetDevice(prev);
    delete t;
    return COS_OK;
}

extern "C" cos_status cos_get_tables_info(const cos_tables *t, cos_tables_info *info) {
    if (!t || !info) {
        cosdp::set_error("cos_get_tables_info: null argument");
        return COS_ERR_ARG;
    }
    memset(info, 0, sizeof *info);
    info->L = t->model.L;
    info->n_tau = t->model.n_tau;
    info->n_flavors = t->model.n_flavors;
    info->symmetric = t->symmetric;
    info->n_mat = t->n_mat;
    info->beta = t->model.beta;
    info->U = t->model.U;
    for (int l = 0; l < COS_MAX_FLAVORS; ++l) info->sigma[l] = t->sigma[l];
    info->d_G = t->d_G;
    info->d_dGdmu = t->d_dG;
    info->bipartite = t->bipartite;
    for (int l = 0; l < COS_MAX_FLAVORS; ++l)
        for (int s = 0; s < 2; ++s) info->sigma2[l][s] = t->sigma2[l][s];
    return COS_OK;
}

extern "C" cos_status cos_copy_table(const cos_tables *t, int which, double *d_dst, cos_stream_t stream) {
    using namespace cosdp;
    if (!t || !d_dst || (which != 0 && which != 1)) {
        set_error("cos_copy_table: bad argument");
        return COS_ERR_ARG;
    }
    if (which == 1 && t->bipartite) {
        set_error("cos_copy_table: honeycomb tables have no dG/dmu table");
        return COS_ERR_ARG;
    }
    if (which == 1) {
        cos_status st = ensure_dtables(const_cast<cos_tables *>(t), (cudaStream_t)stream);
        if (st != COS_OK) return st;
    }
    const size_t n = (size_t)t->n_mat * (t->bipartite ? 4 : 1) * t->model.L * t->model.L * t->model.n_tau;
    cudaError_t e = cudaMemcpyAsync(d_dst, which ? t->d_dG : t->d_G, n * sizeof(double), cudaMemcpyDeviceToDevice,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cos_copy_table");
    return COS_OK;
}
