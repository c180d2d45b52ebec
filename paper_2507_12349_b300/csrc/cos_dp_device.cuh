// Device code shared by the forward and adjoint DP kernels (see cos_dp.cu for the scheme).
#pragma once

#include "cos_internal.h"

namespace cosdp {

static __constant__ uint32_t c_p3[COS_NMAX + 2] = {1u, 3u, 9u, 27u, 81u, 243u, 729u, 2187u, 6561u,
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

// One interaction mask of the forward sweep: every row, the flavor sum of the close, and
// the seed of the next loop (or the sink).  `out` may be null (adjoint recomputation).
template <typename T>
__device__ __forceinline__ void fwd_mask(const OrderTab &tab, uint32_t mask_index, int ell, int n, const T *src,
                                         T *dst1, T *dst2, const T *Ms, const double *Md, int lane, int ci,
                                         int nfl, double sgn, double loop_weight, double sig, bool shifts, bool active,
                                         int lam, int cfg, double *out, int *status) {
    const uint32_t full = (1u << n) - 1u;
    const T negsig = (T)(sgn * sig);
    const uint4 mk = __ldg(reinterpret_cast<const uint4 *>(tab.masks + mask_index));
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
        row_dispatch<T>(__popc(Vrow), src, dst1, dst2, Ms, Md, tab.rank3, Vrow, A, B, J, code, off, h, hidx, nA, n,
                        needclose, shifts, negsig, lane, csum);
    }
    if (!needclose) return;  // no half-visited vertex and not full: disconnected, dropped
    // Flavor sum of the loop-closing weight over the lanes of this configuration.
    double tot = csum;
    if (nfl > 1) {
        const int base = ci * nfl;
        tot = 0.0;
        for (int g = 0; g < nfl; ++g) tot += __shfl_sync(0xFFFFFFFFu, csum, (base + g) & 31);
    }
    const double C = sgn * loop_weight * tot;
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
    } else if (active && lam == 0 && out) {
        const double c = ldexp(C, n - 1);
        out[cfg] = c;
        if (!isfinite(c)) atomicOr(status, kStatusNonFinite);
    }
}

}  // namespace cosdp
