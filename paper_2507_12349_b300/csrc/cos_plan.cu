// CUDA-graph plans and the launch-shape autotuner.
//
// A plan freezes one call (inputs at fixed device addresses) into a CUDA graph: the device
// planner, the gather (coordinates path) and the persistent DP kernel(s).  Creating it runs
// the call once eagerly on the caller's stream to size a private workspace and fix the
// persistent grid, then captures the same launch sequence on a private stream.  Replays are a
// single cudaGraphLaunch with no host-side work.
//
// The autotuner times candidate launch shapes (warps per CTA x CTAs per SM) of the DP kernel
// on synthetic matrices of one order and installs the fastest for that (order, precision,
// lanes per configuration).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "cos_internal.h"

struct cos_plan {
    int device = 0;
    cosdp::Workspace *ws = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int grid = 0;
};

namespace cosdp {

namespace {

template <typename Body>
cos_status make_plan(cudaStream_t stream, Body body, cos_plan **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cos_plan: cudaGetDevice");
    std::string err;
    Workspace *ws = new_private_workspace(dev, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    // 1. eager run: sizes every buffer and fixes the grid
    cos_status st = body(ws, stream);
    if (st == COS_OK) {
        e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) st = cuda_fail(e, "cos_plan: eager run");
    }
    if (st != COS_OK) {
        free_workspace(ws);
        return st;
    }
    ws->fixed_grid = ws->last_grid;
    // 2. capture the same sequence on a private stream
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        free_workspace(ws);
        return cuda_fail(e, "cos_plan: stream");
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = body(ws, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (st == COS_OK && e2 != cudaSuccess) st = cuda_fail(e2, "cos_plan: end capture");
    } else {
        st = cuda_fail(e, "cos_plan: begin capture");
    }
    cudaGraphExec_t exec = nullptr;
    if (st == COS_OK) {
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) st = cuda_fail(e, "cos_plan: instantiate");
    }
    cudaStreamDestroy(cs);
    if (st != COS_OK) {
        if (graph) cudaGraphDestroy(graph);
        free_workspace(ws);
        return st;
    }
    cos_plan *p = new cos_plan();
    p->device = dev;
    p->ws = ws;
    p->graph = graph;
    p->exec = exec;
    p->grid = ws->fixed_grid;
    *out = p;
    return COS_OK;
}

__global__ void fill_matrices_kernel(double *M, size_t count, uint64_t seed) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        // SplitMix64 output of (seed, i), mapped to [-0.9, 0.9): timing inputs only
        uint64_t z = seed * 0x100000000ull + i + 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        M[i] = 1.8 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 0.9;
    }
}

__global__ void fill_layout_kernel(int32_t *order, int64_t *moff, int n_cfg, int n, int64_t stride) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cfg; c += gridDim.x * blockDim.x) {
        order[c] = n;
        moff[c] = (int64_t)c * stride;
    }
}

}  // namespace
}  // namespace cosdp

using namespace cosdp;

extern "C" cos_status cos_plan_create_batch(const cos_tables *t, int n_cfg, int n_max, const int32_t *d_order,
                                            const int64_t *d_offset, const int32_t *d_site, const double *d_tau,
                                            cos_precision precision, double *d_out, double *d_abs_mass,
                                            cos_stream_t stream, cos_plan **out) {
    if (!out) {
        set_error("cos_plan_create_batch: null out");
        return COS_ERR_ARG;
    }
    *out = nullptr;
    cos_status st = check_batch(t, n_cfg, n_max, d_order, d_offset, d_site, d_tau, precision, d_out,
                                "cos_plan_create_batch");
    if (st != COS_OK) return st;
    if (n_cfg == 0) {
        set_error("cos_plan_create_batch: empty batch");
        return COS_ERR_ARG;
    }
    return make_plan((cudaStream_t)stream,
                     [&](Workspace *ws, cudaStream_t s) {
                         return batch_body(ws, t, n_cfg, n_max, d_order, d_offset, d_site, d_tau, precision, d_out,
                                           d_abs_mass, s);
                     },
                     out);
}

extern "C" cos_status cos_plan_create_matrices(int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                                               int n_mat, int loop_weight, const double *h_sigma, const double *d_M,
                                               cos_precision precision, double *d_out, double *d_abs_mass,
                                               cos_stream_t stream, cos_plan **out) {
    if (!out) {
        set_error("cos_plan_create_matrices: null out");
        return COS_ERR_ARG;
    }
    *out = nullptr;
    cos_status st = check_matrices(n_cfg, n_max, d_order, d_moff, n_mat, loop_weight, d_M, precision, d_out,
                                   "cos_plan_create_matrices");
    if (st != COS_OK) return st;
    if (n_cfg == 0) {
        set_error("cos_plan_create_matrices: empty batch");
        return COS_ERR_ARG;
    }
    std::vector<double> sig(n_mat, 0.0);
    if (h_sigma) sig.assign(h_sigma, h_sigma + n_mat);
    return make_plan((cudaStream_t)stream,
                     [&](Workspace *ws, cudaStream_t s) {
                         return matrices_body(ws, n_cfg, n_max, d_order, d_moff, n_mat, loop_weight,
                                              h_sigma ? sig.data() : nullptr, d_M, precision, d_out, d_abs_mass, s);
                     },
                     out);
}

extern "C" cos_status cos_plan_launch(cos_plan *p, cos_stream_t stream) {
    if (!p || !p->exec) {
        set_error("cos_plan_launch: null plan");
        return COS_ERR_ARG;
    }
    cudaError_t e = cudaGraphLaunch(p->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cos_plan_launch");
    return COS_OK;
}

extern "C" cos_status cos_plan_status(cos_plan *p, cos_stream_t stream) {
    if (!p) {
        set_error("cos_plan_status: null plan");
        return COS_ERR_ARG;
    }
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cos_plan_status");
    int word = 0;
    e = cudaMemcpy(&word, p->ws->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(p->ws->status, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "cos_plan_status read");
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

extern "C" cos_status cos_plan_grid(const cos_plan *p, int *grid) {
    if (!p || !grid) {
        set_error("cos_plan_grid: null argument");
        return COS_ERR_ARG;
    }
    *grid = p->grid;
    return COS_OK;
}

extern "C" cos_status cos_plan_destroy(cos_plan *p) {
    if (!p) return COS_OK;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    free_workspace(p->ws);
    delete p;
    return COS_OK;
}

extern "C" cos_status cos_set_tuning(int n, cos_precision precision, int n_mat, int warps, int ctas_per_sm,
                                     int prefetch) {
    if (n < 1 || n > COS_NMAX || n_mat < 1 || n_mat > COS_MAX_FLAVORS || warps < 1 ||
        warps > (precision == COS_FP64 ? 16 : 20) ||
        ctas_per_sm < 1 || ctas_per_sm > 8 || (precision != COS_FP64 && precision != COS_MIXED && precision != COS_DF64)) {
        set_error("cos_set_tuning: out of range");
        return COS_ERR_ARG;
    }
    Tuning t;
    t.warps = warps;
    t.ctas_per_sm = ctas_per_sm;
    t.prefetch = prefetch < 0 ? 0 : (prefetch > 4 ? 4 : prefetch);
    set_tuning(n, precision, n_mat, t);
    return COS_OK;
}

extern "C" cos_status cos_get_tuning(int n, cos_precision precision, int n_mat, int *warps, int *ctas_per_sm,
                                     int *prefetch) {
    if (n < 1 || n > COS_NMAX || !warps || !ctas_per_sm) {
        set_error("cos_get_tuning: bad argument");
        return COS_ERR_ARG;
    }
    const Tuning t = get_tuning(n, precision, n_mat);
    *warps = t.warps;
    *ctas_per_sm = t.ctas_per_sm;
    if (prefetch) *prefetch = t.prefetch;
    return COS_OK;
}

extern "C" cos_status cos_autotune(int n, int n_mat, int loop_weight, int shifts, cos_precision precision,
                                   int n_cfg, cos_stream_t stream, int *best_warps, int *best_ctas,
                                   int *best_prefetch, double *best_ms) {
    if (n < 1 || n > COS_NMAX || n_mat < 1 || n_mat > COS_MAX_FLAVORS || loop_weight < 1 || n_cfg < 1 ||
        (precision != COS_FP64 && precision != COS_MIXED && precision != COS_DF64)) {
        set_error("cos_autotune: out of range");
        return COS_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    std::string err;
    Workspace *ws = new_private_workspace(dev, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    const int64_t stride = (int64_t)n_mat * n * n;
    double *M = nullptr, *outb = nullptr;
    int32_t *order = nullptr;
    int64_t *moff = nullptr;
    cudaError_t e = cudaMalloc(&M, sizeof(double) * stride * n_cfg);
    if (e == cudaSuccess) e = cudaMalloc(&outb, sizeof(double) * n_cfg);
    if (e == cudaSuccess) e = cudaMalloc(&order, sizeof(int32_t) * n_cfg);
    if (e == cudaSuccess) e = cudaMalloc(&moff, sizeof(int64_t) * n_cfg);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    cos_status st = COS_OK;
    if (e != cudaSuccess) st = cuda_fail(e, "cos_autotune: buffers");
    std::vector<double> sig(n_mat, shifts ? 0.05 : 0.0);
    Tuning best;
    double best_t = 1e300;
    const Tuning before = get_tuning(n, precision, n_mat);
    if (st == COS_OK) {
        fill_matrices_kernel<<<256, 256, 0, s>>>(M, (size_t)stride * n_cfg, 12345u + n);
        fill_layout_kernel<<<64, 256, 0, s>>>(order, moff, n_cfg, n, stride);
        const size_t smem = dp_smem_bytes(precision, n);
        // candidates: every (warps, ctas) the occupancy calculator admits, with prefetch into L2;
        // then the best shape again with prefetch off, into L1, and (mixed, double-float) one row ahead
        std::vector<Tuning> cands;
        const int warp_c[] = {2, 4, 8, 10, 12, 16, 20};
        const int cta_c[] = {1, 2, 3, 4};
        for (int w : warp_c)
            for (int c : cta_c)
                if ((w <= 16 || precision != COS_FP64) && dp_max_active_ctas(precision, w * 32, smem) >= c) {
                    Tuning cand;
                    cand.warps = w;
                    cand.ctas_per_sm = c;
                    cand.prefetch = 1;
                    cands.push_back(cand);
                }
        auto time_one = [&](const Tuning &cand, double *t_out) -> cos_status {
            set_tuning(n, precision, n_mat, cand);
            ws->fixed_grid = 0;
            cos_status s2 = matrices_body(ws, n_cfg, n, order, moff, n_mat, loop_weight, sig.data(), M, precision,
                                          outb, nullptr, s);
            double t = 1e300;
            for (int rep = 0; rep < 2 && s2 == COS_OK; ++rep) {
                cudaEventRecord(e0, s);
                s2 = matrices_body(ws, n_cfg, n, order, moff, n_mat, loop_weight, sig.data(), M, precision, outb,
                                   nullptr, s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                t = std::min(t, (double)ms);
            }
            *t_out = t;
            return s2;
        };
        for (const Tuning &cand : cands) {
            double t = 0.0;
            st = time_one(cand, &t);
            if (st != COS_OK) break;
            if (t < best_t) {
                best_t = t;
                best = cand;
            }
        }
        if (st == COS_OK && best_t < 1e300) {
            const Tuning shape = best;
            for (int pf : {0, 2, 3, 4}) {
                if (pf >= 3 && precision == COS_FP64) continue;   // row-ahead: the pair kernels' modes
                Tuning alt = shape;
                alt.prefetch = pf;
                double t = 0.0;
                st = time_one(alt, &t);
                if (st != COS_OK) break;
                if (t < best_t) {
                    best_t = t;
                    best = alt;
                }
            }
        }
    }
    if (st == COS_OK && best_t < 1e300) {
        set_tuning(n, precision, n_mat, best);
        if (const char *path = getenv("COS_TUNE_OUT")) {
            if (FILE *f = fopen(path, "a")) {
                fprintf(f, "%d %d %d %d %d %.4f %d\n", n, (int)precision, n_mat, best.warps, best.ctas_per_sm, best_t,
                        best.prefetch);
                fclose(f);
            }
        }
        if (best_warps) *best_warps = best.warps;
        if (best_ctas) *best_ctas = best.ctas_per_sm;
        if (best_prefetch) *best_prefetch = best.prefetch;
        if (best_ms) *best_ms = best_t;
    } else {
        set_tuning(n, precision, n_mat, before);
    }
    cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(M);
    cudaFree(outb);
    cudaFree(order);
    cudaFree(moff);
    free_workspace(ws);
    return st;
}
