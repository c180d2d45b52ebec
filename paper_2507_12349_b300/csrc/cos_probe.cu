// Throughput probes for the roofline denominators: independent FMA chains per thread,
// enough warps to fill every SM sub-partition.  FLOPs = 2 * blocks * threads * chains * iters.
#include <algorithm>

#include "cos_internal.h"

namespace cosdp {

template <typename T, int CHAINS>
__global__ void fma_probe_kernel(int iters, T *sink) {
    T a[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) a[c] = (T)(threadIdx.x + c) * (T)1e-3;
    const T b = (T)0.999999, d = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) a[c] = a[c] * b + d;   // contracted to one FMA
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += a[c];
    if (s == (T)-1.2345) sink[blockIdx.x] = s;   // never true; keeps the chains live
}

}  // namespace cosdp

extern "C" cos_status cos_peak_probe(int kind, int blocks, int threads, int iters, void *d_sink, cos_stream_t stream) {
    using namespace cosdp;
    if (blocks < 1 || threads < 32 || threads > 1024 || iters < 1 || !d_sink || kind < 0 || kind > 4) {
        set_error("cos_peak_probe: bad argument");
        return COS_ERR_ARG;
    }
    // kind 0/1: FP64 / FP32 with the default chains; kind 2..4: FP64 with 4, 16, 32 chains
    // (a sweep over instruction-level parallelism for the peak search).
    cudaStream_t s = (cudaStream_t)stream;
    switch (kind) {
        case 0: fma_probe_kernel<double, 8><<<blocks, threads, 0, s>>>(iters, (double *)d_sink); break;
        case 1: fma_probe_kernel<float, 16><<<blocks, threads, 0, s>>>(iters, (float *)d_sink); break;
        case 2: fma_probe_kernel<double, 4><<<blocks, threads, 0, s>>>(iters, (double *)d_sink); break;
        case 3: fma_probe_kernel<double, 16><<<blocks, threads, 0, s>>>(iters, (double *)d_sink); break;
        case 4: fma_probe_kernel<double, 32><<<blocks, threads, 0, s>>>(iters, (double *)d_sink); break;
        default: break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "cos_peak_probe");
    return COS_OK;
}

// Verification hook for the integer-pipe FP32 <-> FP64 conversions of the mixed-precision DP
// (widen / narrow_to in cos_dp_device.cuh): applies them elementwise so tests can compare
// them bit for bit with the conversion instructions.
#include "cos_dp_device.cuh"

namespace cosdp {
__global__ void convert_check_kernel(int64_t n, const double *in64, const float *in32, float *narrowed,
                                     double *widened) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        narrowed[i] = narrow_to(0.0f, in64[i]);
        widened[i] = widen(in32[i]);
    }
}
}  // namespace cosdp

extern "C" cos_status cos_convert_check(int64_t n, const double *d_in64, const float *d_in32, float *d_narrowed,
                                        double *d_widened, cos_stream_t stream) {
    using namespace cosdp;
    if (n < 0 || (n > 0 && (!d_in64 || !d_in32 || !d_narrowed || !d_widened))) {
        set_error("cos_convert_check: bad argument");
        return COS_ERR_ARG;
    }
    if (n == 0) return COS_OK;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    convert_check_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(n, d_in64, d_in32, d_narrowed, d_widened);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "cos_convert_check");
    return COS_OK;
}
