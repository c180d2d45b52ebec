// Measurement and verification instruments used by the benchmark and the tests.  They are
// built into their own library (libcos_instr.so) beside libcos.so and are not part of the
// library's interface: nothing in libcos calls them, and include/ declares none of them.
//
//   cos_instr_fma_probe     independent FMA chains per thread (enough warps to fill every SM
//                           sub-partition): the measured throughput of the FP64 / FP32 pipes
//                           that the benchmark reports beside the unit-count peaks.
//   cos_instr_row_traffic   scattered 512-byte rows (each lane 16 bytes), read and written at
//                           pseudo-random row indices of two buffers: the DRAM rate that the
//                           DP kernels' state traffic pattern sustains at a given number of
//                           warps and rows in flight per warp.
//   cos_instr_convert_check applies the integer-pipe FP32 <-> FP64 conversions of the mixed
//                           precision DP (widen / narrow_to of cos_dp_device.cuh, the very
//                           device functions the kernels inline) elementwise, so that a test
//                           can compare them bit for bit with the conversion instructions.
//
// Both return 0 or the CUDA error code of the failed launch (negative for a bad argument).
#include <algorithm>

#include "cos_dp_device.cuh"

namespace cosinstr {

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

__device__ __forceinline__ uint32_t row_hash(uint32_t x) {   // integer finalizer (any good mixer)
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// Each warp, `iters` times: ILP rows read at hashed indices of src, then written at other hashed
// indices of dst (MODE 0), or only read (1) or only written (2).  Indices are < nrows, so every
// access stays inside the nrows * 512 bytes of each buffer.
template <int ILP, int MODE>
__global__ void row_traffic_kernel(const float4 *__restrict__ src, float4 *__restrict__ dst, uint32_t nrows,
                                   int iters, float4 *sink) {
    const int lane = threadIdx.x & 31;
    const uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    float acc = 0.0f;
    for (int it = 0; it < iters; ++it) {
        float4 v[ILP];
        uint32_t w[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            const uint32_t h = row_hash(g * 0x9E3779B9u + (uint32_t)(it * ILP + u) * 0x85EBCA6Bu);
            w[u] = row_hash(h ^ 0x27d4eb2fu) % nrows;
            v[u] = MODE != 2 ? src[(size_t)(h % nrows) * 32 + lane] : make_float4((float)h, 1.0f, 2.0f, 3.0f);
        }
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            if (MODE != 1) dst[(size_t)w[u] * 32 + lane] = v[u];
            else acc += v[u].x;
        }
    }
    if (acc == 1234.5f) sink[0] = make_float4(acc, 0.0f, 0.0f, 0.0f);   // never true; keeps the reads
}

__global__ void convert_check_kernel(int64_t n, const double *in64, const float *in32, float *narrowed,
                                     double *widened) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        narrowed[i] = cosdp::narrow_to(0.0f, in64[i]);
        widened[i] = cosdp::widen(in32[i]);
    }
}

}  // namespace cosinstr

// kind 0 / 1: FP64 / FP32 with 8 / 16 chains per thread; kind 2, 3, 4, 5, 6: FP64 with 4, 16,
// 32, 1, 2 chains (a sweep over instruction-level parallelism; one chain gives the dependent
// issue latency).  Work = 2 * blocks * threads * chains *
// iters flops; d_sink holds `blocks` elements of the probed type.
extern "C" int cos_instr_fma_probe(int kind, int blocks, int threads, int iters, void *d_sink, void *stream) {
    using namespace cosinstr;
    if (blocks < 1 || threads < 32 || threads > 1024 || iters < 1 || !d_sink || kind < 0 || kind > 6) return -1;
    cudaStream_t s = (cudaStream_t)stream;
    switch (kind) {
        case 0: fma_probe_kernel<double, 8><<<blocks, threads, 0, s>>>(iters, (double *)d_sink); break;
        case 1: fma_probe_kernel<float, 16><<<blocks, threads, 0, s>>>(iters, (float *)d_sink); break;
        case 2: fma_probe_kernel<double, 4><<<blocks, threads, 0, s>>>(iters, (double *)d_sink); break;
        case 3: fma_probe_kernel<double, 16><<<blocks, threads, 0, s>>>(iters, (double *)d_sink); break;
        case 4: fma_probe_kernel<double, 32><<<blocks, threads, 0, s>>>(iters, (double *)d_sink); break;
        case 5: fma_probe_kernel<double, 1><<<blocks, threads, 0, s>>>(iters, (double *)d_sink); break;
        default: fma_probe_kernel<double, 2><<<blocks, threads, 0, s>>>(iters, (double *)d_sink); break;
    }
    return (int)cudaGetLastError();
}

// d_narrowed[i] = d_in64[i] rounded to FP32 (nearest even), d_widened[i] = d_in32[i] widened
// to FP64, exactly as the DP kernels compute them.
extern "C" int cos_instr_convert_check(int64_t n, const double *d_in64, const float *d_in32, float *d_narrowed,
                                       double *d_widened, void *stream) {
    using namespace cosinstr;
    if (n < 0 || (n > 0 && (!d_in64 || !d_in32 || !d_narrowed || !d_widened))) return -1;
    if (n == 0) return 0;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    convert_check_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(n, d_in64, d_in32, d_narrowed, d_widened);
    return (int)cudaGetLastError();
}

// Scattered-row traffic: mode 0 read + write, 1 read, 2 write; ilp 1, 4 or 8 rows in flight per
// warp.  d_src and d_dst hold nrows rows of 512 bytes each.  Bytes moved per launch:
// blocks * threads / 32 * iters * ilp * 512 (times 2 in mode 0).
extern "C" int cos_instr_row_traffic(int mode, int ilp, int blocks, int threads, int iters, const void *d_src,
                                     void *d_dst, int64_t nrows, void *stream) {
    using namespace cosinstr;
    if (mode < 0 || mode > 2 || (ilp != 1 && ilp != 4 && ilp != 8) || blocks < 1 || threads < 32 || threads > 1024 ||
        iters < 1 || !d_src || !d_dst || nrows < 1 || nrows > 0xFFFFFFFFll)
        return -1;
    cudaStream_t s = (cudaStream_t)stream;
    const float4 *a = (const float4 *)d_src;
    float4 *b = (float4 *)d_dst;
    const uint32_t r = (uint32_t)nrows;
#define COS_ROWK(I, M)                                                         \
    if (ilp == I && mode == M) row_traffic_kernel<I, M><<<blocks, threads, 0, s>>>(a, b, r, iters, b);
    COS_ROWK(1, 0) COS_ROWK(4, 0) COS_ROWK(8, 0) COS_ROWK(1, 1) COS_ROWK(4, 1) COS_ROWK(8, 1)
    COS_ROWK(1, 2) COS_ROWK(4, 2) COS_ROWK(8, 2)
#undef COS_ROWK
    return (int)cudaGetLastError();
}
