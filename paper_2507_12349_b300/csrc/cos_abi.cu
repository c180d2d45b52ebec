// C ABI of libcos: argument checks, per-(device, stream) workspaces, device status words,
// launch tuning and the public entry points that chain the kernels.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "cos_internal.h"

namespace cosdp {

namespace {
thread_local std::string t_err;
std::mutex g_ws_mu;
std::map<std::pair<int, cudaStream_t>, Workspace *> g_ws;
}  // namespace

void set_error(const std::string &msg) { t_err = msg; }

cos_status cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    cudaGetLastError();  // clear a sticky launch error of this thread
    return e == cudaErrorMemoryAllocation ? COS_ERR_NOMEM : COS_ERR_CUDA;
}

cos_status ensure(void **ptr, size_t *cap, size_t need, size_t elem, const char *what) {
    if (*ptr && *cap >= need) return COS_OK;
    // Growth: the old buffer may still be in use by work queued on this stream.
    cudaDeviceSynchronize();
    cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    const size_t grow = need + need / 4;
    cudaError_t e = cudaMalloc(ptr, grow * elem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(ptr, need * elem);
        if (e != cudaSuccess) {
            *ptr = nullptr;
            return cuda_fail(e, what);
        }
        *cap = need;
        return COS_OK;
    }
    *cap = grow;
    return COS_OK;
}

Workspace *get_workspace(cudaStream_t stream, std::string *err) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_ws_mu);
    auto key = std::make_pair(dev, stream);
    auto it = g_ws.find(key);
    if (it != g_ws.end()) return it->second;
    Workspace *ws = new Workspace();
    ws->device = dev;
    ws->stream = stream;
    e = cudaMalloc(&ws->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ws->plan_counts, 80 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ws->queue, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ws->status, 0, sizeof(int));
    if (e != cudaSuccess) {
        *err = std::string("workspace: ") + cudaGetErrorString(e);
        cudaGetLastError();
        delete ws;
        return nullptr;
    }
    g_ws[key] = ws;
    return ws;
}

// Launch shape per (order, precision, lanes per configuration): warps per CTA and CTAs per SM
// of the persistent grid.  Defaults keep four or more warps per SM sub-partition; large orders
// use one CTA per SM so the layer scratch (two layers of up to 1.26 M slots x 32 lanes at
// n = 12) stays within HBM.  Overrides, in order of precedence: the table filled by
// cos_set_tuning / cos_autotune (and loaded from the file named by COS_TUNE_FILE), then
// COS_TUNE="n:warps:ctas,...".
namespace {
std::mutex g_tune_mu;
std::map<int, Tuning> g_tune;
bool g_tune_loaded = false;
int tune_key(int n, int precision, int nf) { return (n * 4 + precision) * 16 + nf; }

void load_tune_file_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("COS_TUNE_FILE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[256];
    while (fgets(line, sizeof line, f)) {
        int n = 0, prec = 0, nf = 0, w = 0, c = 0, pf = 1;
        double ms = 0.0;
        const int got = sscanf(line, "%d %d %d %d %d %lf %d", &n, &prec, &nf, &w, &c, &ms, &pf);
        if (got >= 5 && n >= 1 && n <= COS_NMAX && w >= 1 && w <= (prec == COS_FP64 ? 16 : 20) && c >= 1 && c <= 8) {
            Tuning t;
            t.warps = w;
            t.ctas_per_sm = c;
            t.prefetch = got >= 7 ? (pf < 0 ? 0 : (pf > 4 ? 4 : pf)) : 1;
            g_tune[tune_key(n, prec, nf)] = t;
        }
    }
    fclose(f);
}
}  // namespace

void set_tuning(int n, int precision, int nf_lanes, Tuning t) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_tune_file_locked();
    g_tune[tune_key(n, precision, nf_lanes)] = t;
}

Tuning get_tuning(int n, int precision, int nf_lanes) {
    Tuning t;
    if (n >= 11) {
        t.warps = 16;
        t.ctas_per_sm = 1;
    } else {
        t.warps = 8;
        t.ctas_per_sm = 2;
    }
    if (const char *s = getenv("COS_TUNE")) {
        const char *p = s;
        while (*p) {
            int tn = 0, tw = 0, tc = 0, used = 0;
            if (sscanf(p, "%d:%d:%d%n", &tn, &tw, &tc, &used) == 3) {
                if (tn == n && tw >= 1 && tw <= 16 && tc >= 1 && tc <= 8) {
                    t.warps = tw;
                    t.ctas_per_sm = tc;
                }
                p += used;
                while (*p == ',' || *p == ' ') ++p;
            } else {
                break;
            }
        }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    load_tune_file_locked();
    auto it = g_tune.find(tune_key(n, precision, nf_lanes));
    if (it != g_tune.end()) t = it->second;
    return t;
}

Workspace *new_private_workspace(int device, std::string *err) {
    Workspace *ws = new Workspace();
    ws->device = device;
    cudaError_t e = cudaMalloc(&ws->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ws->plan_counts, 80 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ws->queue, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ws->status, 0, sizeof(int));
    if (e != cudaSuccess) {
        *err = std::string("workspace: ") + cudaGetErrorString(e);
        cudaGetLastError();
        free_workspace(ws);
        return nullptr;
    }
    return ws;
}

void free_workspace(Workspace *ws) {
    if (!ws) return;
    cudaFree(ws->status);
    cudaFree(ws->plan_counts);
    cudaFree(ws->queue);
    cudaFree(ws->batch_list);
    cudaFree(ws->batches);
    cudaFree(ws->M);
    cudaFree(ws->moff);
    cudaFree(ws->scratch);
    cudaFree(ws->gM);
    cudaFree(ws->gsig);
    cudaFree(ws->sub_order);
    cudaFree(ws->sub_moff);
    cudaFree(ws->sub_key);
    cudaFree(ws->sub_M);
    delete ws;
}

cos_status check_common(int n_cfg, int n_max, cos_precision prec, const char *fn) {
    if (n_cfg < 0) {
        set_error(std::string(fn) + ": n_cfg < 0");
        return COS_ERR_ARG;
    }
    if (n_max < 1 || n_max > COS_NMAX) {
        set_error(std::string(fn) + ": n_max outside [1, 12]");
        return COS_ERR_ORDER;
    }
    if (prec != COS_FP64 && prec != COS_MIXED && prec != COS_DF64) {
        set_error(std::string(fn) + ": unknown precision");
        return COS_ERR_ARG;
    }
    return COS_OK;
}

cos_status run_dp(Workspace *ws, DpLaunch L, double *d_abs_mass, cudaStream_t stream) {
    const int cpb = dp_configs_per_batch(L);
    cos_status st = launch_plan_batches(ws, L.n_cfg, L.n_max, L.order, cpb, stream, L.allow_empty);
    if (st != COS_OK) return st;
    st = launch_dp(ws, L, stream);
    if (st != COS_OK) return st;
    if (d_abs_mass) {
        L.out = d_abs_mass;
        L.absmode = true;
        st = launch_dp(ws, L, stream);
    }
    return st;
}

}  // namespace cosdp

using namespace cosdp;

extern "C" const char *cos_status_string(cos_status s) {
    switch (s) {
        case COS_OK: return "ok";
        case COS_ERR_ARG: return "invalid argument";
        case COS_ERR_ORDER: return "order out of range";
        case COS_ERR_CUDA: return "CUDA error";
        case COS_ERR_TIMEOUT: return "device wait timed out";
        case COS_ERR_NONFINITE: return "non-finite result";
        case COS_ERR_UNIMPLEMENTED: return "not implemented";
        case COS_ERR_NOMEM: return "device memory exhausted";
    }
    return "unknown status";
}

extern "C" const char *cos_last_error(void) { return t_err.c_str(); }

// Frees the workspace of `stream` on the current device after reporting its status (as
// cos_sync_status); the next call on the stream allocates a fresh one.
extern "C" cos_status cos_release_workspace(cos_stream_t stream) {
    const cos_status st = cos_sync_status(stream);
    int dev = 0;
    cudaGetDevice(&dev);
    Workspace *ws = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_ws_mu);
        auto it = g_ws.find(std::make_pair(dev, (cudaStream_t)stream));
        if (it != g_ws.end()) {
            ws = it->second;
            g_ws.erase(it);
        }
    }
    free_workspace(ws);
    return st;
}

extern "C" cos_status cos_sync_status(cos_stream_t stream) {
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cos_sync_status");
    int dev = 0;
    cudaGetDevice(&dev);
    Workspace *ws = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_ws_mu);
        auto it = g_ws.find(std::make_pair(dev, s));
        if (it != g_ws.end()) ws = it->second;
    }
    if (!ws) return COS_OK;
    int word = 0;
    e = cudaMemcpy(&word, ws->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ws->status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "cos_sync_status read");
    if (word & kStatusOrder) {
        set_error("device: order out of range");
        return COS_ERR_ORDER;
    }
    if (word & kStatusSite) {
        set_error("device: site out of range");
        return COS_ERR_ARG;
    }
    if (word & kStatusNonFinite) {
        set_error("device: non-finite result");
        return COS_ERR_NONFINITE;
    }
    return COS_OK;
}

namespace cosdp {
cos_status matrices_body(Workspace *ws, int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                         int n_mat, int loop_weight, const double *h_sigma, const double *d_M,
                         cos_precision precision, double *d_out, double *d_abs_mass, cudaStream_t stream) {
    DpLaunch L;
    L.n_cfg = n_cfg;
    L.n_max = n_max;
    L.order = d_order;
    L.M = d_M;
    L.moff = d_moff;
    L.n_mat = n_mat;
    L.loop_weight = loop_weight;
    for (int l = 0; l < n_mat; ++l) {
        L.sigma[l] = h_sigma ? h_sigma[l] : 0.0;
        if (L.sigma[l] != 0.0) L.shifts = true;
    }
    L.precision = precision;
    L.out = d_out;
    return run_dp(ws, L, d_abs_mass, stream);
}

cos_status check_matrices(int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff, int n_mat,
                          int loop_weight, const double *d_M, cos_precision precision, const double *d_out,
                          const char *fn) {
    cos_status st = check_common(n_cfg, n_max, precision, fn);
    if (st != COS_OK) return st;
    if (n_mat < 1 || n_mat > COS_MAX_FLAVORS || loop_weight < 1) {
        set_error(std::string(fn) + ": n_mat outside [1, 8] or loop_weight < 1");
        return COS_ERR_ARG;
    }
    if (n_cfg > 0 && (!d_order || !d_moff || !d_M || !d_out)) {
        set_error(std::string(fn) + ": null device pointer");
        return COS_ERR_ARG;
    }
    return COS_OK;
}
}  // namespace cosdp

extern "C" cos_status cos_connected_sum_matrices(int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                                                 int n_mat, int loop_weight, const double *h_sigma,
                                                 const double *d_M, cos_precision precision, double *d_out,
                                                 double *d_abs_mass, cos_stream_t stream) {
    cos_status st = check_matrices(n_cfg, n_max, d_order, d_moff, n_mat, loop_weight, d_M, precision, d_out,
                                   "cos_connected_sum_matrices");
    if (st != COS_OK || n_cfg == 0) return st;
    std::string err;
    Workspace *ws = get_workspace((cudaStream_t)stream, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    return matrices_body(ws, n_cfg, n_max, d_order, d_moff, n_mat, loop_weight, h_sigma, d_M, precision, d_out,
                         d_abs_mass, (cudaStream_t)stream);
}

COS_INTERNAL_API cos_status cos_connected_det_matrices(int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                                                 const double *h_alpha, const double *d_M, cos_precision precision,
                                                 double *d_out, double *d_abs_mass, cos_stream_t stream) {
    cos_status st = check_matrices(n_cfg, n_max, d_order, d_moff, 2, 1, d_M, precision, d_out,
                                   "cos_connected_det_matrices");
    if (st != COS_OK || n_cfg == 0) return st;
    std::string err;
    Workspace *ws = get_workspace((cudaStream_t)stream, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    DpLaunch L;
    L.n_cfg = n_cfg;
    L.n_max = n_max;
    L.order = d_order;
    L.M = d_M;
    L.moff = d_moff;
    L.n_mat = 2;
    L.loop_weight = 1;
    for (int b = 0; b < 2; ++b) L.sigma[b] = h_alpha ? h_alpha[b] : 0.0;   // the diagonal shifts
    L.clow = true;
    L.precision = precision;
    L.out = d_out;
    return run_dp(ws, L, d_abs_mass, (cudaStream_t)stream);
}

extern "C" cos_status cos_gather(const cos_tables *t, int n_cfg, const int32_t *d_order, const int64_t *d_offset,
                                 const int32_t *d_site, const double *d_tau, const int64_t *d_moff, double *d_M,
                                 cos_stream_t stream) {
    if (!t || t->bipartite) {
        set_error("cos_gather: null tables, or honeycomb tables (use cos_gather_bipartite)");
        return COS_ERR_ARG;
    }
    if (n_cfg < 0) {
        set_error("cos_gather: n_cfg < 0");
        return COS_ERR_ARG;
    }
    if (n_cfg == 0) return COS_OK;
    if (!d_order || !d_offset || !d_site || !d_tau || !d_moff || !d_M) {
        set_error("cos_gather: null device pointer");
        return COS_ERR_ARG;
    }
    std::string err;
    Workspace *ws = get_workspace((cudaStream_t)stream, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    return launch_gather(t, n_cfg, d_order, d_offset, d_site, d_tau, d_moff, 0, d_M, ws->status,
                         (cudaStream_t)stream);
}

namespace cosdp {
cos_status check_batch(const cos_tables *t, int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_offset,
                       const int32_t *d_site, const double *d_tau, cos_precision precision, const double *d_out,
                       const char *fn) {
    cos_status st = check_common(n_cfg, n_max, precision, fn);
    if (st != COS_OK) return st;
    if (!t || t->bipartite) {
        set_error(std::string(fn) + ": null tables, or honeycomb tables (use the bipartite entry points)");
        return COS_ERR_ARG;
    }
    if (n_cfg > 0 && (!d_order || !d_offset || !d_site || !d_tau || !d_out)) {
        set_error(std::string(fn) + ": null device pointer");
        return COS_ERR_ARG;
    }
    return COS_OK;
}

cos_status batch_body(Workspace *ws, const cos_tables *t, int n_cfg, int n_max, const int32_t *d_order,
                      const int64_t *d_offset, const int32_t *d_site, const double *d_tau, cos_precision precision,
                      double *d_out, double *d_abs_mass, cudaStream_t stream) {
    const int64_t stride = (int64_t)t->n_mat * n_max * n_max;
    cos_status st = ensure((void **)&ws->M, &ws->M_cap, (size_t)n_cfg * stride, sizeof(double), "matrix workspace");
    if (st != COS_OK) return st;
    st = launch_gather(t, n_cfg, d_order, d_offset, d_site, d_tau, nullptr, stride, ws->M, ws->status, stream);
    if (st != COS_OK) return st;
    DpLaunch L;
    L.n_cfg = n_cfg;
    L.n_max = n_max;
    L.order = d_order;
    L.M = ws->M;
    L.moff = nullptr;
    L.mstride = stride;
    L.n_mat = t->n_mat;
    L.loop_weight = t->symmetric ? t->model.n_flavors : 1;
    for (int l = 0; l < t->n_mat; ++l) {
        L.sigma[l] = t->sigma[l];
        if (L.sigma[l] != 0.0) L.shifts = true;
    }
    L.precision = precision;
    L.out = d_out;
    return run_dp(ws, L, d_abs_mass, stream);
}
}  // namespace cosdp

namespace cosdp {
namespace {
// Symmetric SU(2) tables hold one matrix per configuration: copy it into the spin-down block,
// [2][n_c][n_c] at c * stride.
__global__ void dup_spin_block_kernel(int n_cfg, const int32_t *__restrict__ order, int64_t stride,
                                      double *__restrict__ M) {
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_cfg; c += warps) {
        const int n = order[c];
        if (n < 1 || n > COS_NMAX || (int64_t)2 * n * n > stride) continue;
        double *b = M + (int64_t)c * stride;
        for (int e = lane; e < n * n; e += 32) b[n * n + e] = b[e];
    }
}
// dc/dM of a configuration from the stride layout [2][n_c][n_c] at c * stride into the caller's
// blocks at gmoff[c].
__global__ void copy_spin_blocks_kernel(int n_cfg, const int32_t *__restrict__ order, int64_t stride,
                                        const double *__restrict__ src, const int64_t *__restrict__ gmoff,
                                        double *__restrict__ dst) {
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_cfg; c += warps) {
        const int n = order[c];
        if (n < 1 || n > COS_NMAX || (int64_t)2 * n * n > stride) continue;
        for (int e = lane; e < 2 * n * n; e += 32) dst[gmoff[c] + e] = src[(int64_t)c * stride + e];
    }
}

// Collapsed (symmetric) tables: both spin blocks came from one matrix, so dc/dM of that matrix
// is the sum of the two blocks' gradients (folded into block 0 for the chain rule).
__global__ void fold_spin_blocks_kernel(int n_cfg, const int32_t *__restrict__ order, int64_t stride,
                                        double *__restrict__ g) {
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_cfg; c += warps) {
        const int n = order[c];
        if (n < 1 || n > COS_NMAX || (int64_t)2 * n * n > stride) continue;
        double *b = g + (int64_t)c * stride;
        for (int e = lane; e < n * n; e += 32) b[e] += b[n * n + e];
    }
}
}  // namespace
}  // namespace cosdp

COS_INTERNAL_API cos_status cos_connected_det_grad(const cos_tables *t, int n_cfg, int n_max, const int32_t *d_order,
                                             const int64_t *d_offset, const int32_t *d_site, const double *d_tau,
                                             const double *h_alpha, const double *d_gout, double *d_out,
                                             double *d_gM, const int64_t *d_gmoff, double *d_gmu,
                                             double *d_galpha, cos_stream_t stream) {
    const char *fn = "cos_connected_det_grad";
    cos_status st = check_common(n_cfg, n_max, COS_FP64, fn);
    if (st != COS_OK) return st;
    if (!t || t->bipartite || t->model.n_flavors != 2) {
        set_error(std::string(fn) + ": needs SU(2) square-lattice tables (two flavors)");
        return COS_ERR_ARG;
    }
    if (n_cfg == 0) return COS_OK;
    if (!d_order || !d_offset || !d_site || !d_tau || !d_gout || (d_gM && !d_gmoff)) {
        set_error(std::string(fn) + ": null device pointer (d_gM needs d_gmoff)");
        return COS_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::string err;
    Workspace *ws = get_workspace(s, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    if (d_gmu) {
        st = ensure_dtables(const_cast<cos_tables *>(t), s);
        if (st != COS_OK) return st;
    }
    const int64_t stride = (int64_t)2 * n_max * n_max;
    st = ensure((void **)&ws->M, &ws->M_cap, (size_t)n_cfg * stride, sizeof(double), "matrix workspace");
    if (st == COS_OK) st = ensure((void **)&ws->gM, &ws->gM_cap, (size_t)n_cfg * stride, sizeof(double), "gradient workspace");
    if (st == COS_OK) st = ensure((void **)&ws->gsig, &ws->gsig_cap, (size_t)n_cfg * 2, sizeof(double), "alpha gradient");
    if (st != COS_OK) return st;
    st = launch_gather(t, n_cfg, d_order, d_offset, d_site, d_tau, nullptr, stride, ws->M, ws->status, s);
    if (st != COS_OK) return st;
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ws->device);
    const int blocks = std::max(1, std::min((n_cfg * 32 + 255) / 256, 8 * nsm));
    if (t->n_mat == 1) dup_spin_block_kernel<<<blocks, 256, 0, s>>>(n_cfg, d_order, stride, ws->M);
    DpLaunch L;
    L.n_cfg = n_cfg;
    L.n_max = n_max;
    L.order = d_order;
    L.M = ws->M;
    L.moff = nullptr;
    L.mstride = stride;
    L.n_mat = 2;
    L.loop_weight = 1;
    for (int b = 0; b < 2; ++b) L.sigma[b] = h_alpha ? h_alpha[b] : 0.0;
    L.clow = true;
    L.precision = COS_FP64;
    L.out = d_out;
    st = launch_plan_batches(ws, n_cfg, n_max, d_order, kLanes / 2, s);
    if (st != COS_OK) return st;
    st = launch_adjoint(ws, L, d_gout, ws->gM, nullptr, stride, ws->gsig, s);
    if (st != COS_OK) return st;
    if (d_gM) copy_spin_blocks_kernel<<<blocks, 256, 0, s>>>(n_cfg, d_order, stride, ws->gM, d_gmoff, d_gM);
    if (d_galpha) {
        cudaError_t e = cudaMemcpyAsync(d_galpha, ws->gsig, (size_t)n_cfg * 2 * sizeof(double),
                                        cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "alpha gradient copy");
    }
    if (d_gmu) {
        if (t->n_mat == 1) fold_spin_blocks_kernel<<<blocks, 256, 0, s>>>(n_cfg, d_order, stride, ws->gM);
        // dc/dmu_b through the dG/dmu tables (the tables' dispersion shift alpha is 0 here)
        st = launch_chain(t, n_cfg, d_order, d_offset, d_site, d_tau, ws->gM, nullptr, stride, ws->gsig, d_gmu,
                          nullptr, s);
        if (st != COS_OK) return st;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "determinant gradient launches");
    return COS_OK;
}

COS_INTERNAL_API cos_status cos_connected_det_batch(const cos_tables *t, int n_cfg, int n_max, const int32_t *d_order,
                                              const int64_t *d_offset, const int32_t *d_site, const double *d_tau,
                                              const double *h_alpha, cos_precision precision, double *d_out,
                                              double *d_abs_mass, cos_stream_t stream) {
    const char *fn = "cos_connected_det_batch";
    cos_status st = check_batch(t, n_cfg, n_max, d_order, d_offset, d_site, d_tau, precision, d_out, fn);
    if (st != COS_OK) return st;
    if (t->model.n_flavors != 2) {
        set_error(std::string(fn) + ": determinant weights need SU(2) tables (two flavors)");
        return COS_ERR_ARG;
    }
    if (n_cfg == 0) return COS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    std::string err;
    Workspace *ws = get_workspace(s, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    const int64_t stride = (int64_t)2 * n_max * n_max;
    st = ensure((void **)&ws->M, &ws->M_cap, (size_t)n_cfg * stride, sizeof(double), "matrix workspace");
    if (st != COS_OK) return st;
    st = launch_gather(t, n_cfg, d_order, d_offset, d_site, d_tau, nullptr, stride, ws->M, ws->status, s);
    if (st != COS_OK) return st;
    if (t->n_mat == 1) {
        int nsm = 1;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ws->device);
        const int blocks = std::max(1, std::min((n_cfg * 32 + 255) / 256, 8 * nsm));
        dup_spin_block_kernel<<<blocks, 256, 0, s>>>(n_cfg, d_order, stride, ws->M);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "spin block copy launch");
    }
    DpLaunch L;
    L.n_cfg = n_cfg;
    L.n_max = n_max;
    L.order = d_order;
    L.M = ws->M;
    L.moff = nullptr;
    L.mstride = stride;
    L.n_mat = 2;
    L.loop_weight = 1;
    for (int b = 0; b < 2; ++b) L.sigma[b] = h_alpha ? h_alpha[b] : 0.0;   // the diagonal shifts
    L.clow = true;
    L.precision = precision;
    L.out = d_out;
    return run_dp(ws, L, d_abs_mass, s);
}

extern "C" cos_status cos_connected_sum_batch(const cos_tables *t, int n_cfg, int n_max, const int32_t *d_order,
                                              const int64_t *d_offset, const int32_t *d_site, const double *d_tau,
                                              cos_precision precision, double *d_out, double *d_abs_mass,
                                              cos_stream_t stream) {
    cos_status st = check_batch(t, n_cfg, n_max, d_order, d_offset, d_site, d_tau, precision, d_out,
                                "cos_connected_sum_batch");
    if (st != COS_OK || n_cfg == 0) return st;
    std::string err;
    Workspace *ws = get_workspace((cudaStream_t)stream, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    return batch_body(ws, t, n_cfg, n_max, d_order, d_offset, d_site, d_tau, precision, d_out, d_abs_mass,
                      (cudaStream_t)stream);
}

COS_INTERNAL_API cos_status cos_connected_sum_matrices_grad(int n_cfg, int n_max, const int32_t *d_order,
                                                      const int64_t *d_moff, int n_mat, int loop_weight,
                                                      const double *h_sigma, const double *d_M, const double *d_gout,
                                                      double *d_out, double *d_gM, double *d_gsigma,
                                                      cos_stream_t stream) {
    cos_status st = check_common(n_cfg, n_max, COS_FP64, "cos_connected_sum_matrices_grad");
    if (st != COS_OK) return st;
    if (n_mat < 1 || n_mat > COS_MAX_FLAVORS || loop_weight < 1) {
        set_error("cos_connected_sum_matrices_grad: n_mat outside [1, 8] or loop_weight < 1");
        return COS_ERR_ARG;
    }
    if (n_cfg == 0) return COS_OK;
    if (!d_order || !d_moff || !d_M || !d_gout) {
        set_error("cos_connected_sum_matrices_grad: null device pointer");
        return COS_ERR_ARG;
    }
    std::string err;
    Workspace *ws = get_workspace((cudaStream_t)stream, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    DpLaunch L;
    L.n_cfg = n_cfg;
    L.n_max = n_max;
    L.order = d_order;
    L.M = d_M;
    L.moff = d_moff;
    L.n_mat = n_mat;
    L.loop_weight = loop_weight;
    for (int l = 0; l < n_mat; ++l) {
        L.sigma[l] = h_sigma ? h_sigma[l] : 0.0;
        if (L.sigma[l] != 0.0) L.shifts = true;
    }
    L.precision = COS_FP64;
    L.out = d_out;
    st = launch_plan_batches(ws, n_cfg, n_max, d_order, kLanes / n_mat, (cudaStream_t)stream);
    if (st != COS_OK) return st;
    return launch_adjoint(ws, L, d_gout, d_gM, d_moff, 0, d_gsigma, (cudaStream_t)stream);
}

COS_INTERNAL_API cos_status cos_connected_det_matrices_grad(int n_cfg, int n_max, const int32_t *d_order,
                                                      const int64_t *d_moff, const double *h_alpha, const double *d_M,
                                                      const double *d_gout, double *d_out, double *d_gM,
                                                      double *d_galpha, cos_stream_t stream) {
    cos_status st = check_common(n_cfg, n_max, COS_FP64, "cos_connected_det_matrices_grad");
    if (st != COS_OK || n_cfg == 0) return st;
    if (!d_order || !d_moff || !d_M || !d_gout) {
        set_error("cos_connected_det_matrices_grad: null device pointer");
        return COS_ERR_ARG;
    }
    std::string err;
    Workspace *ws = get_workspace((cudaStream_t)stream, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    DpLaunch L;
    L.n_cfg = n_cfg;
    L.n_max = n_max;
    L.order = d_order;
    L.M = d_M;
    L.moff = d_moff;
    L.n_mat = 2;
    L.loop_weight = 1;
    for (int b = 0; b < 2; ++b) L.sigma[b] = h_alpha ? h_alpha[b] : 0.0;   // the diagonal shifts
    L.clow = true;
    L.precision = COS_FP64;
    L.out = d_out;
    st = launch_plan_batches(ws, n_cfg, n_max, d_order, kLanes / 2, (cudaStream_t)stream);
    if (st != COS_OK) return st;
    return launch_adjoint(ws, L, d_gout, d_gM, d_moff, 0, d_galpha, (cudaStream_t)stream);
}

extern "C" cos_status cos_connected_sum_grad(const cos_tables *t, int n_cfg, int n_max, const int32_t *d_order,
                                             const int64_t *d_offset, const int32_t *d_site, const double *d_tau,
                                             const double *d_gout, double *d_out, double *d_gM,
                                             const int64_t *d_gmoff, double *d_gmu, double *d_galpha,
                                             cos_stream_t stream) {
    cos_status st = check_common(n_cfg, n_max, COS_FP64, "cos_connected_sum_grad");
    if (st != COS_OK) return st;
    if (!t || t->bipartite) {
        set_error("cos_connected_sum_grad: null tables, or honeycomb tables (no bipartite gradient)");
        return COS_ERR_ARG;
    }
    if (n_cfg == 0) return COS_OK;
    if (!d_order || !d_offset || !d_site || !d_tau || !d_gout || (d_gM && !d_gmoff)) {
        set_error("cos_connected_sum_grad: null device pointer (d_gM needs d_gmoff)");
        return COS_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::string err;
    Workspace *ws = get_workspace(s, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    if (d_gmu || d_galpha) {
        st = ensure_dtables(const_cast<cos_tables *>(t), s);
        if (st != COS_OK) return st;
    }
    const int64_t stride = (int64_t)t->n_mat * n_max * n_max;
    st = ensure((void **)&ws->M, &ws->M_cap, (size_t)n_cfg * stride, sizeof(double), "matrix workspace");
    if (st != COS_OK) return st;
    double *gM = d_gM;
    const int64_t *gmoff = d_gmoff;
    int64_t gmstride = 0;
    if (!gM) {
        st = ensure((void **)&ws->gM, &ws->gM_cap, (size_t)n_cfg * stride, sizeof(double), "gradient workspace");
        if (st != COS_OK) return st;
        gM = ws->gM;
        gmstride = stride;
    }
    st = ensure((void **)&ws->gsig, &ws->gsig_cap, (size_t)n_cfg * t->n_mat, sizeof(double), "sigma gradient");
    if (st != COS_OK) return st;
    st = launch_gather(t, n_cfg, d_order, d_offset, d_site, d_tau, nullptr, stride, ws->M, ws->status, s);
    if (st != COS_OK) return st;
    DpLaunch L;
    L.n_cfg = n_cfg;
    L.n_max = n_max;
    L.order = d_order;
    L.M = ws->M;
    L.moff = nullptr;
    L.mstride = stride;
    L.n_mat = t->n_mat;
    L.loop_weight = t->symmetric ? t->model.n_flavors : 1;
    for (int l = 0; l < t->n_mat; ++l) {
        L.sigma[l] = t->sigma[l];
        if (L.sigma[l] != 0.0) L.shifts = true;
    }
    L.precision = COS_FP64;
    L.out = d_out;
    st = launch_plan_batches(ws, n_cfg, n_max, d_order, kLanes / t->n_mat, s);
    if (st != COS_OK) return st;
    // the adjoint writes dM with the gather's stride layout unless the caller gave offsets
    st = launch_adjoint(ws, L, d_gout, gM, gmoff, gmstride, ws->gsig, s);
    if (st != COS_OK) return st;
    if (d_gmu || d_galpha)
        st = launch_chain(t, n_cfg, d_order, d_offset, d_site, d_tau, gM, gmoff, gmstride, ws->gsig, d_gmu, d_galpha,
                          s);
    return st;
}
