// Honeycomb two-band propagator tables and the bipartite gather.
//
// Methods A, honeycomb lattice: per flavor l the Bloch Hamiltonian on the sublattices (A, B)
//   H_l(k) = [[d - m, eps(k)], [conj(eps(k)), -d - m]],  d = delta_l, m = mu_l - alpha_l,
//   eps(k) = -t (1 + exp(i k1) + exp(i k2)),  k1 = 2 pi m_1 / L, k2 = 2 pi m_2 / L,
// and G_l(R, tau) = -(1/L^2) sum_k exp(i k.R) exp(-H tau)(1 - n_F(H)) for 0 < tau < beta.
// A 2 x 2 Hermitian matrix function is f(H) = (f+ + f-)/2 + (f+ - f-)/(2 r) (H + m), with
// eigenvalues E+- = -m +- r, r = sqrt(d^2 + |eps|^2) (H + m is traceless): no eigenvector
// routine is needed.  The real-space hopping is real, so G is real:
//   G_AA = -(1/L^2) sum_k cos(k.R) (W0 + d Wg),   G_BB = ... (W0 - d Wg),
//   G_AB = -(1/L^2) sum_k Wg (cos(k.R) Re eps - sin(k.R) Im eps),
//   G_BA = -(1/L^2) sum_k Wg (cos(k.R) Re eps + sin(k.R) Im eps),
// W0 = (f+ + f-)/2, Wg = (f+ - f-)/(2 r) (0 when r = 0, where f+ = f-), f = exp(-E tau)(1 - n_F(E)).
// Tables: [n_mat][s][t][R][m], R = r1 + L r2 (cell coordinates), tau_m = m beta / (n_tau - 1).
#include <cmath>
#include <cstring>
#include <string>

#include "cos_internal.h"

namespace cosdp {

namespace {

// exp(-E tau)(1 - n_F(E)) in the overflow-free form of each sign of E.
__device__ __forceinline__ double tau_w(double E, double tau, double beta) {
    if (E >= 0.0) return exp(-E * tau) / (1.0 + exp(-beta * E));
    return exp(E * (beta - tau)) / (1.0 + exp(beta * E));
}

// n_F(E) = 1 / (1 + exp(beta E)), overflow-free.
__device__ __forceinline__ double fermi(double E, double beta) {
    if (E >= 0.0) {
        const double x = exp(-beta * E);
        return x / (1.0 + x);
    }
    return 1.0 / (1.0 + exp(beta * E));
}

// W0, Wg for every (matrix, momentum, tau point), and eps(k) (Re, Im) per momentum.
// deriv: their derivatives with respect to mu instead.  E = -m +- r with m = mu - alpha, so
// d f(E) / d mu = -f'(E) = f(E) (tau - beta n_F(E)); d and eps(k), hence r, do not depend on mu.
__global__ void hc_weight_kernel(int L, int n_mat, int n_tau, double t, double beta, const double *dm,
                                 double *W0, double *Wg, double *eps_re, double *eps_im, int deriv) {
    const int LL = L * L;
    const size_t total = (size_t)n_mat * LL * n_tau;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(i % n_tau);
        const int k = (int)((i / n_tau) % LL);
        const int l = (int)(i / ((size_t)n_tau * LL));
        const int m1 = k % L, m2 = k / L;
        const double re = -t * (1.0 + cospi(2.0 * m1 / L) + cospi(2.0 * m2 / L));
        const double im = -t * (sinpi(2.0 * m1 / L) + sinpi(2.0 * m2 / L));
        const double d = dm[2 * l], mm = dm[2 * l + 1];
        const double r = sqrt(d * d + re * re + im * im);
        const double tau = beta * m / (n_tau - 1);
        double fp = tau_w(-mm + r, tau, beta), fm = tau_w(-mm - r, tau, beta);
        if (deriv) {
            fp *= tau - beta * fermi(-mm + r, beta);
            fm *= tau - beta * fermi(-mm - r, beta);
        }
        W0[i] = 0.5 * (fp + fm);
        Wg[i] = r > 0.0 ? (fp - fm) / (2.0 * r) : 0.0;
        if (l == 0 && m == 0) {
            eps_re[k] = re;
            eps_im[k] = im;
        }
    }
}

// G[l][s][t][R][m] by the momentum sum; cos/sin(k.R) = cos/sin(2 pi ((m1 r1 + m2 r2) mod L) / L).
__global__ void hc_ksum_kernel(int L, int n_mat, int n_tau, const double *dm, const double *W0, const double *Wg,
                               const double *eps_re, const double *eps_im, double *G) {
    extern __shared__ double s_lut[];   // cos, sin of 2 pi q / L
    for (int q = threadIdx.x; q < L; q += blockDim.x) {
        s_lut[q] = cospi(2.0 * q / L);
        s_lut[L + q] = sinpi(2.0 * q / L);
    }
    __syncthreads();
    const int LL = L * L;
    const size_t total = (size_t)n_mat * 4 * LL * n_tau;
    const double scale = -1.0 / (double)LL;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(i % n_tau);
        const int R = (int)((i / n_tau) % LL);
        const int st = (int)((i / ((size_t)n_tau * LL)) % 4);
        const int l = (int)(i / ((size_t)n_tau * LL * 4));
        const int r1 = R % L, r2 = R / L;
        const double d = dm[2 * l];
        const double *w0 = W0 + (size_t)l * LL * n_tau + m;
        const double *wg = Wg + (size_t)l * LL * n_tau + m;
        double acc = 0.0;
        for (int m2 = 0; m2 < L; ++m2) {
            const int q2 = (m2 * r2) % L;
            for (int m1 = 0; m1 < L; ++m1) {
                const int k = m1 + L * m2;
                const int q = (m1 * r1 + q2) % L;
                const double c = s_lut[q], s = s_lut[L + q];
                const double a0 = w0[(size_t)k * n_tau], ag = wg[(size_t)k * n_tau];
                double term;
                if (st == 0) term = c * fma(d, ag, a0);
                else if (st == 3) term = c * fma(-d, ag, a0);
                else if (st == 1) term = ag * (c * eps_re[k] - s * eps_im[k]);
                else term = ag * (c * eps_re[k] + s * eps_im[k]);
                acc += term;
            }
        }
        G[i] = scale * acc;
    }
}

// One warp per configuration: M4[l][(i,s)][(j,t)] = G_l^{st}(R_i - R_j, tau_i - tau_j).
__global__ void hc_gather_kernel(const double *__restrict__ G, int L, int n_tau, double beta, int n_mat, int n_cfg,
                                 const int32_t *__restrict__ order, const int64_t *__restrict__ offset,
                                 const int32_t *__restrict__ site, const double *__restrict__ tau,
                                 const int64_t *__restrict__ moff, double *__restrict__ M, int *status) {
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int LL = L * L;
    const double scale = (double)(n_tau - 1) / beta;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_cfg; c += warps) {
        const int n = order[c];
        // a negative offset marks an order above the caller's n_max (its slot would overflow)
        if (n < 1 || n > COS_BIP_NMAX || moff[c] < 0) {
            if (lane == 0) atomicOr(status, kStatusOrder);
            continue;
        }
        const int64_t o = offset[c];
        double *Mc = M + moff[c];
        const int n2 = 2 * n, nn = n2 * n2;
        for (int e = lane; e < n_mat * nn; e += 32) {
            const int l = e / nn, rr = (e / n2) % n2, cc = e % n2;
            const int i = rr >> 1, s = rr & 1, j = cc >> 1, tt = cc & 1;
            const int si = site[o + i], sj = site[o + j];
            if (si < 0 || si >= LL || sj < 0 || sj >= LL) {
                atomicOr(status, kStatusSite);
                Mc[e] = nan("");
                continue;
            }
            const int d1 = ((si % L) - (sj % L) + L) % L;
            const int d2 = ((si / L) - (sj / L) + L) % L;
            const int R = d1 + L * d2;
            const double dt = tau[o + i] - tau[o + j];
            double sg = 1.0, tv = dt;
            if (dt <= 0.0) {
                sg = -1.0;
                tv = dt + beta;
            }
            const double x = tv * scale;
            int m = (int)floor(x);
            m = max(0, min(m, n_tau - 2));
            const double f = x - m;
            const double *row = G + ((((size_t)l * 2 + s) * 2 + tt) * LL + R) * n_tau + m;
            Mc[e] = sg * fma(f, row[1] - row[0], row[0]);
        }
    }
}

// deriv: the dG/dmu tables (into d_dG) instead of G.
cos_status build_hc_tables(cos_tables *t, cudaStream_t stream, bool deriv = false) {
    const int L = t->model.L, LL = L * L, n_tau = t->model.n_tau, n_mat = t->n_mat;
    const size_t nW = (size_t)n_mat * LL * n_tau;
    double *d_dm = nullptr, *d_W0 = nullptr, *d_Wg = nullptr, *d_er = nullptr, *d_ei = nullptr;
    double h_dm[2 * COS_MAX_FLAVORS];
    for (int l = 0; l < n_mat; ++l) {
        h_dm[2 * l] = t->delta[l];
        h_dm[2 * l + 1] = t->mu[l] - t->alpha[l];
    }
    cudaError_t e = cudaMalloc(&d_dm, sizeof(double) * 2 * n_mat);
    if (e == cudaSuccess) e = cudaMalloc(&d_W0, sizeof(double) * nW);
    if (e == cudaSuccess) e = cudaMalloc(&d_Wg, sizeof(double) * nW);
    if (e == cudaSuccess) e = cudaMalloc(&d_er, sizeof(double) * LL);
    if (e == cudaSuccess) e = cudaMalloc(&d_ei, sizeof(double) * LL);
    double **dst = deriv ? &t->d_dG : &t->d_G;
    if (e == cudaSuccess) e = cudaMalloc(dst, sizeof(double) * nW * 4);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_dm, h_dm, sizeof(double) * 2 * n_mat, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) {
        const int wb = (int)std::min<size_t>((nW + 255) / 256, 65535);
        hc_weight_kernel<<<wb, 256, 0, stream>>>(L, n_mat, n_tau, t->model.t, t->model.beta, d_dm, d_W0, d_Wg, d_er,
                                                 d_ei, deriv ? 1 : 0);
        const int kb = (int)std::min<size_t>((4 * nW + 255) / 256, 65535);
        hc_ksum_kernel<<<kb, 256, 2 * L * sizeof(double), stream>>>(L, n_mat, n_tau, d_dm, d_W0, d_Wg, d_er, d_ei,
                                                                     *dst);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    cudaFree(d_dm);
    cudaFree(d_W0);
    cudaFree(d_Wg);
    cudaFree(d_er);
    cudaFree(d_ei);
    if (e != cudaSuccess) {
        if (deriv) {   // no half-built derivative table is left behind for a later call
            cudaFree(t->d_dG);
            t->d_dG = nullptr;
        }
        return cuda_fail(e, "honeycomb tables");
    }
    return COS_OK;
}

cos_status launch_gather_bip(const cos_tables *t, int n_cfg, const int32_t *order, const int64_t *offset,
                             const int32_t *site, const double *tau, const int64_t *moff, double *M, int *status,
                             cudaStream_t stream) {
    if (n_cfg == 0) return COS_OK;
    const int threads = 256;
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, t->device);
    const int blocks = std::max(1, std::min((n_cfg * 32 + threads - 1) / threads, 8 * nsm));
    hc_gather_kernel<<<blocks, threads, 0, stream>>>(t->d_G, t->model.L, t->model.n_tau, t->model.beta, t->n_mat,
                                                      n_cfg, order, offset, site, tau, moff, M, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "bipartite gather launch");
    return COS_OK;
}

}  // namespace

// Device work of the coordinates path: per-configuration matrix offsets, gather, DP.
// Slot offsets of the batch entry's own matrix layout (stride = the slot of order n_max); -1 for
// an order outside [1, n_max], which the gather then skips and flags.
__global__ void hc_moff_kernel(int n_cfg, int n_max, const int32_t *order, int64_t *moff, int64_t stride) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cfg; c += gridDim.x * blockDim.x)
        moff[c] = (order[c] >= 1 && order[c] <= n_max) ? (int64_t)c * stride : -1;
}

// Chain rule through the honeycomb tables, one warp per configuration:
//   dc/dmu_l = sum over (i,s),(j,t) of dc/dM4_l[(i,s)][(j,t)] dG_l^{st}/dmu (the gather's
//   interpolation of the dG/dmu table), and dc/dalpha_l = -(that sum) + (dc/dsigma_{l,A} +
//   dc/dsigma_{l,B}) / U, since sigma_{l,A/B} = (alpha_l +- delta_l) / U and G depends on mu - alpha.
// Collapsed (symmetric) tables: the common derivative split evenly over the flavors.
__global__ void hc_chain_kernel(const double *__restrict__ dG, int L, int n_tau, double beta, int n_mat,
                                int n_flavors, int symmetric, double U, int n_cfg, const int32_t *__restrict__ order,
                                const int64_t *__restrict__ offset, const int32_t *__restrict__ site,
                                const double *__restrict__ tau, const double *__restrict__ gM,
                                const int64_t *__restrict__ moff, const double *__restrict__ gsig2,
                                double *__restrict__ gmu, double *__restrict__ galpha) {
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int LL = L * L;
    const double scale = (double)(n_tau - 1) / beta;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_cfg; c += warps) {
        const int n = order[c];
        if (n < 1 || n > COS_BIP_NMAX || moff[c] < 0) continue;
        const int64_t o = offset[c];
        const int n2 = 2 * n, nn = n2 * n2;
        const double *g = gM + moff[c];
        for (int l = 0; l < n_mat; ++l) {
            double acc = 0.0;
            for (int e = lane; e < nn; e += 32) {
                const int rr = e / n2, cc = e % n2;
                const int i = rr >> 1, s = rr & 1, j = cc >> 1, tt = cc & 1;
                const int si = site[o + i], sj = site[o + j];
                if (si < 0 || si >= LL || sj < 0 || sj >= LL) continue;
                const int d1 = ((si % L) - (sj % L) + L) % L;
                const int d2 = ((si / L) - (sj / L) + L) % L;
                const double dt = tau[o + i] - tau[o + j];
                double sg = 1.0, tv = dt;
                if (dt <= 0.0) {
                    sg = -1.0;
                    tv = dt + beta;
                }
                const double x = tv * scale;
                int m = (int)floor(x);
                m = max(0, min(m, n_tau - 2));
                const double f = x - m;
                const double *row = dG + ((((size_t)l * 2 + s) * 2 + tt) * LL + d1 + L * d2) * n_tau + m;
                acc = fma(g[(size_t)l * nn + e], sg * fma(f, row[1] - row[0], row[0]), acc);
            }
            for (int w = 16; w >= 1; w >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, w);
            if (lane == 0) {
                const double gs = gsig2 ? gsig2[((int64_t)c * n_mat + l) * 2] + gsig2[((int64_t)c * n_mat + l) * 2 + 1]
                                        : 0.0;
                if (symmetric) {
                    for (int q = 0; q < n_flavors; ++q) {
                        if (gmu) gmu[(int64_t)c * n_flavors + q] = acc / n_flavors;
                        if (galpha) galpha[(int64_t)c * n_flavors + q] = (-acc + gs / U) / n_flavors;
                    }
                } else {
                    if (gmu) gmu[(int64_t)c * n_flavors + l] = acc;
                    if (galpha) galpha[(int64_t)c * n_flavors + l] = -acc + gs / U;
                }
            }
        }
    }
}

// dc/dM4 from the entry's stride layout (moff) into the caller's blocks at gmoff.
__global__ void hc_copy_blocks_kernel(int n_cfg, int n_mat, const int32_t *order, const int64_t *moff,
                                      const double *src, const int64_t *gmoff, double *dst) {
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_cfg; c += warps) {
        const int n = order[c];
        if (n < 1 || n > COS_BIP_NMAX || moff[c] < 0) continue;
        const int cnt = n_mat * 4 * n * n;
        for (int e = lane; e < cnt; e += 32) dst[gmoff[c] + e] = src[moff[c] + e];
    }
}

// Collapsed (symmetric) tables serve both spin blocks: copy block 0 ([2n][2n]) into block 1.
__global__ void hc_dup_block_kernel(int n_cfg, const int32_t *order, const int64_t *moff, double *M) {
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_cfg; c += warps) {
        const int n = order[c];
        if (n < 1 || n > COS_BIP_NMAX || moff[c] < 0) continue;
        const int nn = 4 * n * n;
        double *b = M + moff[c];
        for (int e = lane; e < nn; e += 32) b[nn + e] = b[e];
    }
}

// Collapsed tables: both spin blocks came from one matrix, so its gradient is the blocks' sum
// (folded into block 0 for the chain rule).
__global__ void hc_fold_block_kernel(int n_cfg, const int32_t *order, const int64_t *moff, double *g) {
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_cfg; c += warps) {
        const int n = order[c];
        if (n < 1 || n > COS_BIP_NMAX || moff[c] < 0) continue;
        const int nn = 4 * n * n;
        double *b = g + moff[c];
        for (int e = lane; e < nn; e += 32) b[e] += b[nn + e];
    }
}

}  // namespace cosdp

using namespace cosdp;

extern "C" cos_status cos_build_propagators_honeycomb(const cos_honeycomb_model *m, cos_stream_t stream,
                                                      cos_tables **out) {
    if (!m || !out) {
        set_error("cos_build_propagators_honeycomb: null argument");
        return COS_ERR_ARG;
    }
    *out = nullptr;
    if (m->L < 1 || m->L > 128 || m->n_tau < 2 || m->n_tau > 65536 || m->n_flavors < 1 ||
        m->n_flavors > COS_MAX_FLAVORS || !(m->beta > 0.0) || m->U == 0.0 || !m->mu || !m->alpha || !m->delta) {
        set_error("cos_build_propagators_honeycomb: model out of range");
        return COS_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cos_tables *t = new cos_tables();
    t->device = dev;
    t->bipartite = 1;
    t->mu.assign(m->mu, m->mu + m->n_flavors);
    t->alpha.assign(m->alpha, m->alpha + m->n_flavors);
    t->delta.assign(m->delta, m->delta + m->n_flavors);
    t->model.L = m->L;
    t->model.t = m->t;
    t->model.beta = m->beta;
    t->model.U = m->U;
    t->model.n_flavors = m->n_flavors;
    t->model.mu = t->mu.data();
    t->model.alpha = t->alpha.data();
    t->model.n_tau = m->n_tau;
    bool sym = true;
    for (int l = 1; l < m->n_flavors; ++l)
        if (t->mu[l] != t->mu[0] || t->alpha[l] != t->alpha[0] || t->delta[l] != t->delta[0]) sym = false;
    t->symmetric = sym ? 1 : 0;
    t->n_mat = sym ? 1 : m->n_flavors;
    for (int l = 0; l < COS_MAX_FLAVORS; ++l) {
        const bool in = l < m->n_flavors;
        t->sigma[l] = in ? t->alpha[l] / m->U : 0.0;
        t->sigma2[l][0] = in ? (t->alpha[l] + t->delta[l]) / m->U : 0.0;   // sublattice A
        t->sigma2[l][1] = in ? (t->alpha[l] - t->delta[l]) / m->U : 0.0;   // sublattice B
    }
    t->d_G = nullptr;
    t->d_dG = nullptr;
    cos_status st = build_hc_tables(t, (cudaStream_t)stream);
    if (st != COS_OK) {
        cudaFree(t->d_G);
        delete t;
        return st;
    }
    *out = t;
    return COS_OK;
}

extern "C" cos_status cos_gather_bipartite(const cos_tables *t, int n_cfg, const int32_t *d_order,
                                           const int64_t *d_offset, const int32_t *d_site, const double *d_tau,
                                           const int64_t *d_moff, double *d_M4, cos_stream_t stream) {
    if (!t || !t->bipartite) {
        set_error("cos_gather_bipartite: tables missing or not bipartite");
        return COS_ERR_ARG;
    }
    if (n_cfg < 0 || (n_cfg > 0 && (!d_order || !d_offset || !d_site || !d_tau || !d_moff || !d_M4))) {
        set_error("cos_gather_bipartite: bad argument");
        return COS_ERR_ARG;
    }
    if (n_cfg == 0) return COS_OK;
    std::string err;
    Workspace *ws = get_workspace((cudaStream_t)stream, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    return launch_gather_bip(t, n_cfg, d_order, d_offset, d_site, d_tau, d_moff, d_M4, ws->status,
                             (cudaStream_t)stream);
}

COS_INTERNAL_API cos_status cos_connected_sum_bipartite_batch(const cos_tables *t, int n_cfg, int n_max,
                                                        const int32_t *d_order, const int64_t *d_offset,
                                                        const int32_t *d_site, const double *d_tau,
                                                        cos_precision precision, double *d_out, double *d_abs_mass,
                                                        cos_stream_t stream) {
    const char *fn = "cos_connected_sum_bipartite_batch";
    if (!t || !t->bipartite) {
        set_error(std::string(fn) + ": tables missing or not bipartite");
        return COS_ERR_ARG;
    }
    if (n_cfg < 0) {
        set_error(std::string(fn) + ": n_cfg < 0");
        return COS_ERR_ARG;
    }
    if (n_max < 1 || n_max > COS_BIP_NMAX) {
        set_error(std::string(fn) + ": n_max outside [1, 9]");
        return COS_ERR_ORDER;
    }
    if (precision != COS_FP64 && precision != COS_MIXED && precision != COS_DF64) {
        set_error(std::string(fn) + ": unknown precision");
        return COS_ERR_ARG;
    }
    if (n_cfg == 0) return COS_OK;
    if (!d_order || !d_offset || !d_site || !d_tau || !d_out) {
        set_error(std::string(fn) + ": null device pointer");
        return COS_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::string err;
    Workspace *ws = get_workspace(s, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    const int n_mat = t->n_mat;
    const int64_t stride = (int64_t)n_mat * 4 * n_max * n_max;
    cos_status st = ensure((void **)&ws->M, &ws->M_cap, (size_t)n_cfg * stride, sizeof(double), "bipartite matrices");
    if (st == COS_OK) st = ensure((void **)&ws->moff, &ws->moff_cap, (size_t)n_cfg, sizeof(int64_t), "matrix offsets");
    if (st != COS_OK) return st;
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ws->device);
    hc_moff_kernel<<<std::max(1, std::min((n_cfg + 255) / 256, 8 * nsm)), 256, 0, s>>>(n_cfg, n_max, d_order,
                                                                                       ws->moff, stride);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "bipartite offsets");
    st = launch_gather_bip(t, n_cfg, d_order, d_offset, d_site, d_tau, ws->moff, ws->M, ws->status, s);
    if (st != COS_OK) return st;
    double sig2[2 * COS_MAX_FLAVORS];
    for (int l = 0; l < n_mat; ++l) {
        sig2[2 * l] = t->sigma2[l][0];
        sig2[2 * l + 1] = t->sigma2[l][1];
    }
    const int loop_weight = t->symmetric ? t->model.n_flavors : 1;
    return bip_matrices_body(ws, n_cfg, n_max, d_order, ws->moff, n_mat, loop_weight, sig2, ws->M, precision, d_out,
                             d_abs_mass, s);
}

COS_INTERNAL_API cos_status cos_connected_det_bipartite_batch(const cos_tables *t, int n_cfg, int n_max,
                                                        const int32_t *d_order, const int64_t *d_offset,
                                                        const int32_t *d_site, const double *d_tau,
                                                        const double *h_alpha2, cos_precision precision,
                                                        double *d_out, double *d_abs_mass, cos_stream_t stream) {
    const char *fn = "cos_connected_det_bipartite_batch";
    if (!t || !t->bipartite || t->model.n_flavors != 2) {
        set_error(std::string(fn) + ": needs two-flavor (spin up, spin down) honeycomb tables");
        return COS_ERR_ARG;
    }
    if (n_cfg < 0) {
        set_error(std::string(fn) + ": n_cfg < 0");
        return COS_ERR_ARG;
    }
    if (n_max < 1 || n_max > COS_BIP_NMAX) {
        set_error(std::string(fn) + ": n_max outside [1, 9]");
        return COS_ERR_ORDER;
    }
    if (precision != COS_FP64 && precision != COS_MIXED && precision != COS_DF64) {
        set_error(std::string(fn) + ": unknown precision");
        return COS_ERR_ARG;
    }
    if (n_cfg == 0) return COS_OK;
    if (!d_order || !d_offset || !d_site || !d_tau || !d_out) {
        set_error(std::string(fn) + ": null device pointer");
        return COS_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::string err;
    Workspace *ws = get_workspace(s, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    const int64_t stride = (int64_t)2 * 4 * n_max * n_max;   // two spin blocks per configuration
    cos_status st = ensure((void **)&ws->M, &ws->M_cap, (size_t)n_cfg * stride, sizeof(double), "bipartite matrices");
    if (st == COS_OK) st = ensure((void **)&ws->moff, &ws->moff_cap, (size_t)n_cfg, sizeof(int64_t), "matrix offsets");
    if (st != COS_OK) return st;
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ws->device);
    const int blocks = std::max(1, std::min((n_cfg + 255) / 256, 8 * nsm));
    hc_moff_kernel<<<blocks, 256, 0, s>>>(n_cfg, n_max, d_order, ws->moff, stride);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "bipartite offsets");
    st = launch_gather_bip(t, n_cfg, d_order, d_offset, d_site, d_tau, ws->moff, ws->M, ws->status, s);
    if (st != COS_OK) return st;
    if (t->n_mat == 1) {
        const int wblocks = std::max(1, std::min((n_cfg * 32 + 255) / 256, 8 * nsm));
        hc_dup_block_kernel<<<wblocks, 256, 0, s>>>(n_cfg, d_order, ws->moff, ws->M);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "spin block copy");
    }
    return bip_matrices_body(ws, n_cfg, n_max, d_order, ws->moff, 2, 1, h_alpha2, ws->M, precision, d_out,
                             d_abs_mass, s, true);
}

COS_INTERNAL_API cos_status cos_connected_sum_bipartite_grad(const cos_tables *t, int n_cfg, int n_max,
                                                       const int32_t *d_order, const int64_t *d_offset,
                                                       const int32_t *d_site, const double *d_tau,
                                                       const double *d_gout, double *d_out, double *d_gM4,
                                                       const int64_t *d_gmoff, double *d_gmu, double *d_galpha,
                                                       cos_stream_t stream) {
    const char *fn = "cos_connected_sum_bipartite_grad";
    if (!t || !t->bipartite) {
        set_error(std::string(fn) + ": tables missing or not bipartite");
        return COS_ERR_ARG;
    }
    if (n_cfg < 0) {
        set_error(std::string(fn) + ": n_cfg < 0");
        return COS_ERR_ARG;
    }
    if (n_max < 1 || n_max > COS_BIP_NMAX) {
        set_error(std::string(fn) + ": n_max outside [1, 9]");
        return COS_ERR_ORDER;
    }
    if (n_cfg == 0) return COS_OK;
    if (!d_order || !d_offset || !d_site || !d_tau || !d_gout || (d_gM4 && !d_gmoff)) {
        set_error(std::string(fn) + ": null device pointer (d_gM4 needs d_gmoff)");
        return COS_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::string err;
    Workspace *ws = get_workspace(s, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    cos_tables *tm = const_cast<cos_tables *>(t);
    if ((d_gmu || d_galpha) && !tm->d_dG) {
        cos_status st = build_hc_tables(tm, s, true);
        if (st != COS_OK) return st;
    }
    const int n_mat = t->n_mat;
    const int64_t stride = (int64_t)n_mat * 4 * n_max * n_max;
    cos_status st = ensure((void **)&ws->M, &ws->M_cap, (size_t)n_cfg * stride, sizeof(double), "bipartite matrices");
    if (st == COS_OK) st = ensure((void **)&ws->moff, &ws->moff_cap, (size_t)n_cfg, sizeof(int64_t), "matrix offsets");
    if (st == COS_OK) st = ensure((void **)&ws->gM, &ws->gM_cap, (size_t)n_cfg * stride, sizeof(double), "gradient");
    if (st == COS_OK)
        st = ensure((void **)&ws->gsig, &ws->gsig_cap, (size_t)n_cfg * n_mat * 2, sizeof(double), "shift gradient");
    if (st != COS_OK) return st;
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ws->device);
    hc_moff_kernel<<<std::max(1, std::min((n_cfg + 255) / 256, 8 * nsm)), 256, 0, s>>>(n_cfg, n_max, d_order,
                                                                                       ws->moff, stride);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "bipartite offsets");
    st = launch_gather_bip(t, n_cfg, d_order, d_offset, d_site, d_tau, ws->moff, ws->M, ws->status, s);
    if (st != COS_OK) return st;
    double sig2[2 * COS_MAX_FLAVORS];
    for (int l = 0; l < n_mat; ++l) {
        sig2[2 * l] = t->sigma2[l][0];
        sig2[2 * l + 1] = t->sigma2[l][1];
    }
    const int loop_weight = t->symmetric ? t->model.n_flavors : 1;
    st = bip_grad_dp(fn, n_cfg, n_max, d_order, ws->moff, n_mat, loop_weight, sig2, ws->M, d_gout, d_out, ws->gM,
                     ws->gsig, s);
    if (st != COS_OK) return st;
    const int wblocks = std::max(1, std::min((n_cfg * 32 + 255) / 256, 8 * nsm));
    if (d_gM4) hc_copy_blocks_kernel<<<wblocks, 256, 0, s>>>(n_cfg, n_mat, d_order, ws->moff, ws->gM, d_gmoff, d_gM4);
    if (d_gmu || d_galpha)
        hc_chain_kernel<<<wblocks, 256, 0, s>>>(t->d_dG, t->model.L, t->model.n_tau, t->model.beta, n_mat,
                                                 t->model.n_flavors, t->symmetric, t->model.U, n_cfg, d_order,
                                                 d_offset, d_site, d_tau, ws->gM, ws->moff, ws->gsig, d_gmu, d_galpha);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "bipartite chain rule launches");
    return COS_OK;
}

COS_INTERNAL_API cos_status cos_connected_det_bipartite_grad(const cos_tables *t, int n_cfg, int n_max,
                                                       const int32_t *d_order, const int64_t *d_offset,
                                                       const int32_t *d_site, const double *d_tau,
                                                       const double *h_alpha2, const double *d_gout, double *d_out,
                                                       double *d_gM4, const int64_t *d_gmoff, double *d_gmu,
                                                       double *d_galpha2, cos_stream_t stream) {
    const char *fn = "cos_connected_det_bipartite_grad";
    if (!t || !t->bipartite || t->model.n_flavors != 2) {
        set_error(std::string(fn) + ": needs two-flavor (spin up, spin down) honeycomb tables");
        return COS_ERR_ARG;
    }
    if (n_cfg < 0) {
        set_error(std::string(fn) + ": n_cfg < 0");
        return COS_ERR_ARG;
    }
    if (n_max < 1 || n_max > COS_BIP_NMAX) {
        set_error(std::string(fn) + ": n_max outside [1, 9]");
        return COS_ERR_ORDER;
    }
    if (n_cfg == 0) return COS_OK;
    if (!d_order || !d_offset || !d_site || !d_tau || !d_gout || (d_gM4 && !d_gmoff)) {
        set_error(std::string(fn) + ": null device pointer (d_gM4 needs d_gmoff)");
        return COS_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::string err;
    Workspace *ws = get_workspace(s, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    cos_tables *tm = const_cast<cos_tables *>(t);
    if (d_gmu && !tm->d_dG) {
        cos_status st = build_hc_tables(tm, s, true);
        if (st != COS_OK) return st;
    }
    const int64_t stride = (int64_t)2 * 4 * n_max * n_max;   // two spin blocks per configuration
    cos_status st = ensure((void **)&ws->M, &ws->M_cap, (size_t)n_cfg * stride, sizeof(double), "bipartite matrices");
    if (st == COS_OK) st = ensure((void **)&ws->moff, &ws->moff_cap, (size_t)n_cfg, sizeof(int64_t), "matrix offsets");
    if (st == COS_OK) st = ensure((void **)&ws->gM, &ws->gM_cap, (size_t)n_cfg * stride, sizeof(double), "gradient");
    if (st == COS_OK) st = ensure((void **)&ws->gsig, &ws->gsig_cap, (size_t)n_cfg * 4, sizeof(double), "alpha gradient");
    if (st != COS_OK) return st;
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ws->device);
    hc_moff_kernel<<<std::max(1, std::min((n_cfg + 255) / 256, 8 * nsm)), 256, 0, s>>>(n_cfg, n_max, d_order,
                                                                                       ws->moff, stride);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "bipartite offsets");
    st = launch_gather_bip(t, n_cfg, d_order, d_offset, d_site, d_tau, ws->moff, ws->M, ws->status, s);
    if (st != COS_OK) return st;
    const int wblocks = std::max(1, std::min((n_cfg * 32 + 255) / 256, 8 * nsm));
    if (t->n_mat == 1) hc_dup_block_kernel<<<wblocks, 256, 0, s>>>(n_cfg, d_order, ws->moff, ws->M);
    st = bip_grad_dp(fn, n_cfg, n_max, d_order, ws->moff, 2, 1, h_alpha2, ws->M, d_gout, d_out, ws->gM, ws->gsig, s,
                     true);
    if (st != COS_OK) return st;
    if (d_gM4) hc_copy_blocks_kernel<<<wblocks, 256, 0, s>>>(n_cfg, 2, d_order, ws->moff, ws->gM, d_gmoff, d_gM4);
    if (d_galpha2) {
        e = cudaMemcpyAsync(d_galpha2, ws->gsig, (size_t)n_cfg * 4 * sizeof(double), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "alpha gradient copy");
    }
    if (d_gmu) {
        if (t->n_mat == 1) hc_fold_block_kernel<<<wblocks, 256, 0, s>>>(n_cfg, d_order, ws->moff, ws->gM);
        // dc/dmu_b through the dG/dmu tables; the tables' own shift weights play no part here
        hc_chain_kernel<<<wblocks, 256, 0, s>>>(t->d_dG, t->model.L, t->model.n_tau, t->model.beta, t->n_mat, 2,
                                                 t->symmetric, t->model.U, n_cfg, d_order, d_offset, d_site, d_tau,
                                                 ws->gM, ws->moff, nullptr, d_gmu, nullptr);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "determinant gradient launches");
    return COS_OK;
}
