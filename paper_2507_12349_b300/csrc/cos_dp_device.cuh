// Device code shared by the forward and adjoint DP kernels (see cos_dp.cu for the scheme).
#pragma once

#include "cos_df64.cuh"
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
    int prefetch;               // prefetch the next mask's states: 0 off, 1 into L2, 2 into L1 (tuned)
    double *csub;               // nullable (all-subsets mode): connected sums c(S), see csub_key
    const int64_t *csub_key;    // per configuration: (base << 4) | shift; c(S) of its vertex set S
                                // (bit i = vertex i) goes to csub[base + (S << shift)]
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

// Conversions of the FP64 inputs to a state or matrix element type (once per batch).
__device__ __forceinline__ void to_elem(double x, double &r) { r = x; }
__device__ __forceinline__ void to_elem(double x, float &r) { r = (float)x; }
__device__ __forceinline__ void to_elem(double x, df64 &r) { r = df64_from(x); }

// Exact FP32 -> FP64 widening by bit manipulation (IEEE-754 binary32 / binary64 layouts: the
// exponent is rebiased by 1023 - 127 = 896 and the 23-bit fraction moves up by 29 bits).  On
// B300 the FP64 conversion instruction occupies the FP64 pipe; this keeps the widening on the
// integer pipe.  Zeros are handled by integer selects; subnormals, infinities and NaNs go
// through the conversion instruction in a separate (non-inlined) function, so the compiler
// cannot turn the rare path into a predicated conversion on every lane.  Results equal the
// conversion instruction's in every case.
static __device__ __noinline__ double widen_slow(float f) { return (double)f; }
__device__ __forceinline__ double widen(double x) { return x; }
__device__ __forceinline__ double widen(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    const uint32_t frac = u & 0x7FFFFFu;
    uint32_t hi = (u & 0x80000000u) | ((e + 896u) << 20) | (frac >> 3);
    uint32_t lo = frac << 29;
    if (e == 0u) {
        hi = u & 0x80000000u;
        lo = 0u;
    }
    double d = __hiloint2double((int)hi, (int)lo);
    if (__builtin_expect((e == 0u && frac != 0u) || e == 0xFFu, 0)) d = widen_slow(f);
    return d;
}

// FP64 -> FP32 with round-to-nearest-even on the integer pipe for results in the normal
// float range (the 52-bit fraction keeps its top 23 bits, the 29 dropped bits decide the
// rounding, a carry moves into the exponent); zeros by integer selects; results that would
// be subnormal, infinite or NaN take the conversion instruction (non-inlined, rare).
static __device__ __noinline__ float narrow_slow(double x) { return (float)x; }
__device__ __forceinline__ float narrow_to(float, double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32);
    const uint32_t sgn = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu) - 896;          // binary32 biased exponent
    const uint32_t mant = (uint32_t)((b >> 29) & 0x7FFFFFull);
    const uint32_t rem = (uint32_t)(b & 0x1FFFFFFFull);
    uint32_t r = sgn | ((uint32_t)e << 23) | mant;
    r += (rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u))) ? 1u : 0u;
    const bool zero = (b << 1) == 0ull;
    if (zero) r = sgn;
    float f = __uint_as_float(r);
    if (__builtin_expect(!zero && (e < 1 || e > 254), 0)) f = narrow_slow(x);
    return f;
}
__device__ __forceinline__ double narrow_to(double, double x) { return x; }

__device__ __forceinline__ double close_value(double a) { return a; }
__device__ __forceinline__ double close_value(const DotAcc &a) { return widen(a.s) + widen(a.c); }

// Loop-closing accumulators.  FP64 states close in FP64 (one FMA per state).  FP32 states (the
// mixed mode) close with a compensated FP32 dot product (Ogita, Rump and Oishi, "Accurate sum
// and dot product", SIAM J. Sci. Comput. 26 (2005), Dot2): the close matrices are split into
// FP32 pairs hi + lo, each term o (hi + lo) adds its leading product with TwoSum and collects
// the product's exact error (FMA TwoProduct) and the cross term o lo in a second FP32 sum.  The
// pair (s, c) is widened exactly and added in FP64 once per mask.  Error of a mask's close:
// at most gamma_N^2 sum |terms| (N terms, gamma_N = N 2^-24 / (1 - N 2^-24)) plus 2^-47 sum
// |terms| for the matrices' split and the cross terms, so the cancelling close keeps about 47
// bits while every operation stays on the FP32 pipe (the mixed mode's FP32 extension states
// carry 2^-24 relative errors of their own).
template <typename T>
struct CloseAcc {
    using type = double;
};
template <>
struct CloseAcc<float> {
    using type = DotAcc;
};
__device__ __forceinline__ void close_init(double &a) { a = 0.0; }
__device__ __forceinline__ void close_init(DotAcc &a) { a.s = a.c = 0.0f; }
__device__ __forceinline__ void close_add(double &acc, double o, double m) { acc = fma(o, m, acc); }
__device__ __forceinline__ void close_add(DotAcc &acc, float o, df64 m) {
    const float p = __fmul_rn(o, m.hi);
    float e = __fmaf_rn(o, m.hi, -p);   // o hi - p exactly
    e = __fmaf_rn(o, m.lo, e);          // plus the cross term
    float t;
    acc.s = two_sum(acc.s, p, t);
    acc.c = __fadd_rn(acc.c, __fadd_rn(e, t));
}

// close_add for two configurations at once (packed FP32, the same operations per component).
__device__ __forceinline__ void close_add2(DotAcc2 &acc, float2 o, float2 mhi, float2 mlo) {
    const float2 p = mul2(o, mhi);
    float2 e = fma2(o, mhi, neg2(p));
    e = fma2(o, mlo, e);
    float2 t;
    acc.s = two_sum2(acc.s, p, t);
    acc.c = add2(acc.c, add2(e, t));
}

// -x by flipping the sign bit (integer pipe; FP64 instructions are the scarce resource).
__device__ __forceinline__ double neg(double x) {
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

// Sum of v over the nfl lanes of configuration ci (lanes ci*nfl .. ci*nfl+nfl-1), identical
// bits in every lane of the group: a butterfly for powers of two (log2 nfl additions; each
// level adds the same two values in every lane), a fixed-order chain otherwise.
__device__ __forceinline__ double flavor_sum(double v, int nfl, int ci) {
    if (nfl == 1) return v;
    if ((nfl & (nfl - 1)) == 0) {
        for (int o = 1; o < nfl; o <<= 1) {
            const double w = __shfl_xor_sync(0xFFFFFFFFu, v, o);
            const bool upper = (threadIdx.x & o) != 0;
            const double lo = upper ? w : v, hi = upper ? v : w;   // operand selects, one add
            v = lo + hi;
        }
        return v;
    }
    const int base = ci * nfl;
    double t = __shfl_sync(0xFFFFFFFFu, v, base & 31);
    for (int g = 1; g < nfl; ++g) t += __shfl_sync(0xFFFFFFFFu, v, (base + g) & 31);
    return t;
}

// Prefetches the state block of a mask (its |H| x |A| slots of 32 lanes), one cache line per
// lane and instruction: level 1 = into L2, level 2 = into L1 as well.
template <typename T>
__device__ __forceinline__ void prefetch_block(const T *src, uint32_t off, uint32_t nslots, int lane, int level) {
    for (uint32_t s = lane; s < nslots; s += kLanes) {
        const char *p = reinterpret_cast<const char *>(src + (size_t)(off + s) * kLanes);
        if (level >= 2) {
            asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
            if (sizeof(T) == 8) asm volatile("prefetch.global.L1 [%0];" ::"l"(p + 128));
        } else {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
            if (sizeof(T) == 8) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + 128));
        }
    }
}

// Extension targets of one mask, computed once per mask with one lane per target and read
// back with shuffles by every row of the mask.  Lane q (q < popc(J)) holds the q-th
// extension mu -> mu + e_j:
//   off1 : block offset of mask mu + e_j in the next layer
//   meta : ai1 (bits 0-3, slot of endpoint j inside a row of that block), nA1 (4-7, row
//          length), untouched (8, mu_j = 0), j (12-15), H1 (16-27, heads of mu + e_j)
struct TgtInfo {
    uint32_t off1, meta;
};

__device__ __forceinline__ TgtInfo mask_targets(uint32_t A, uint32_t B, uint32_t J, uint32_t code,
                                                const uint32_t *__restrict__ rank3, int lane) {
    TgtInfo ti = {0u, 0u};
    if (lane < __popc(J)) {
        const int j = __fns(J, 0, lane + 1);
        const uint32_t bj = 1u << j;
        const bool untouched = !(A & bj);
        const uint32_t A1 = A | bj;
        const uint32_t B1 = untouched ? B : (B | bj);
        const uint32_t nA1 = (uint32_t)__popc(A1);
        const uint32_t ai1 = (uint32_t)__popc(A1 & (bj - 1u));
        ti.off1 = __ldg(rank3 + code + c_p3[j]);
        ti.meta = ai1 | (nA1 << 4) | ((untouched ? 1u : 0u) << 8) | ((uint32_t)j << 12) |
                  (head_set(B1, A1 & ~B1) << 16);
    }
    return ti;
}

// Store of one extension's dot product into its target slot.  Every target has exactly one
// writer: shift points enter through the shifted diagonal of the extension matrices (see
// cos_dp.cu), so no target is read back and accumulated -- except the seed of a new loop at
// vertex 0, which the same thread adds after the row (fwd_mask).
template <typename T>
__device__ __forceinline__ void push_target(T *__restrict__ dst1, const TgtInfo &ti, int q, T d, uint32_t hlow,
                                            int lane) {
    const uint32_t off1 = __shfl_sync(0xFFFFFFFFu, ti.off1, q);
    const uint32_t meta = __shfl_sync(0xFFFFFFFFu, ti.meta, q);
    const uint32_t ai1 = meta & 15u, nA1 = (meta >> 4) & 15u;
    const uint32_t hi1 = (uint32_t)__popc((meta >> 16) & hlow);
    dst1[(size_t)(off1 + hi1 * nA1 + ai1) * kLanes + lane] = d;
}

// One row (mu, h): load its NV endpoint states, accumulate the close, push every extension.
template <typename T, int NV, typename CM, typename CA>
__device__ __forceinline__ void do_row(const T *__restrict__ src, T *__restrict__ dst1, const T *__restrict__ Ms,
                                       const CM *__restrict__ Md, const TgtInfo &ti, int nJ, uint32_t J,
                                       uint32_t Vrow, uint32_t A, uint32_t off, int h, int hidx, int nA, int n,
                                       bool needclose, int lane, CA &csum) {
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
        for (int t = 0; t < NV; ++t) close_add(csum, o[t], Md[vs[t] + h * kLanes]);
    }
    const uint32_t hlow = (1u << h) - 1u;
    uint32_t jj = J;
    int q = 0;
    // extensions two at a time: two independent FMA chains in flight per row
    for (; q + 1 < nJ; q += 2) {
        const int ja = __ffs(jj) - 1;
        jj &= jj - 1u;
        const int jb = __ffs(jj) - 1;
        jj &= jj - 1u;
        T da = T(0), db = T(0);
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            da = Prec<T>::fma_(o[t], Ms[vs[t] + ja * kLanes], da);
            db = Prec<T>::fma_(o[t], Ms[vs[t] + jb * kLanes], db);
        }
        push_target(dst1, ti, q, da, hlow, lane);
        push_target(dst1, ti, q + 1, db, hlow, lane);
    }
    if (q < nJ) {
        const int j = __ffs(jj) - 1;
        T d = T(0);
#pragma unroll
        for (int t = 0; t < NV; ++t) d = Prec<T>::fma_(o[t], Ms[vs[t] + j * kLanes], d);
        push_target(dst1, ti, q, d, hlow, lane);
    }
}

template <typename T, typename CM, typename CA>
__device__ __forceinline__ void row_dispatch(int nv, const T *src, T *dst1, const T *Ms, const CM *Md,
                                             const TgtInfo &ti, int nJ, uint32_t J, uint32_t Vrow, uint32_t A,
                                             uint32_t off, int h, int hidx, int nA, int n, bool needclose, int lane,
                                             CA &csum) {
#define COS_ROW(K)                                                                                            \
    case K:                                                                                                   \
        do_row<T, K>(src, dst1, Ms, Md, ti, nJ, J, Vrow, A, off, h, hidx, nA, n, needclose, lane, csum);       \
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
// Ms: extension matrices (shifted diagonal); Md: FP64 close matrices times sgn * w.
// SUBSETS: also close the masks with no half-visited vertex and store c(S) (all-subsets mode);
// `csub` is this lane's output base (valid on active lanes), `cshift` the root's bit offset.
// CLOW: determinant weights without cycle factors (Alg. 1, see cos_dp.cu): lanes are the two
// spin blocks, the first loop never steps onto vertex 0, its close opens the next loop in the
// spin-down block only, and the sink takes no 2^(n-1).
template <typename T, bool SUBSETS = false, bool CLOW = false, typename CM = double>
__device__ __forceinline__ void fwd_mask(const OrderTab &tab, uint32_t mask_index, uint32_t next_index, int ell,
                                         int n, const T *src, T *dst1, const T *Ms, const CM *Md, int lane,
                                         int ci, int nfl, double sgn, double sig, bool shifts, bool active, int lam,
                                         int cfg, double *out, int *status, int prefetch, double *csub = nullptr,
                                         int cshift = 0) {
    const uint32_t full = (1u << n) - 1u;
    const uint4 mk = __ldg(reinterpret_cast<const uint4 *>(tab.masks + mask_index));
    const uint32_t A = mk.x & 0xFFFFu, B = mk.x >> 16, code = mk.y, off = mk.z;
    const uint32_t ones = A & ~B;
    const uint32_t H = head_set(B, ones);
    // (CLOW: while the first loop is open, vertex 0 holds its head point and is no target)
    const uint32_t J = full & ~B & (CLOW ? ~(ones & 1u) : 0xFFFFFFFFu);
    const int nA = __popc(A);
    // Closes feed a new loop (a half-visited vertex remains) or the sink (all full).  With no
    // half-visited vertex and untouched ones left, the cover of S = {mu_i = 2} is complete and
    // connected: its close is c(S) (times 2^(1-|S|)), kept only in the all-subsets mode.
    const bool dead = (ones == 0u) && (B != full);
    const bool needclose = !dead || SUBSETS;
    if (prefetch > 0 && next_index != 0xFFFFFFFFu) {
        // the next mask of this warp in the layer: start its loads while this one computes
        const uint4 nk = __ldg(reinterpret_cast<const uint4 *>(tab.masks + next_index));
        const uint32_t nA_ = nk.x & 0xFFFFu, nB_ = nk.x >> 16;
        prefetch_block(src, nk.z, (uint32_t)(__popc(head_set(nB_, nA_ & ~nB_)) * __popc(nA_)), lane, prefetch);
    }
    typename CloseAcc<T>::type csum;
    close_init(csum);
    const TgtInfo ti = mask_targets(A, B, J, code, tab.rank3, lane);
    const int nJ = __popc(J);
    for (uint32_t hh = H; hh; hh &= hh - 1u) {
        const int h = __ffs(hh) - 1;
        const int hidx = __popc(H & ((1u << h) - 1u));
        const uint32_t Vrow = row_vmask(A, ones, h);
        row_dispatch<T>(__popc(Vrow), src, dst1, Ms, Md, ti, nJ, J, Vrow, A, off, h, hidx, nA, n, needclose, lane,
                        csum);
    }
    if (!needclose) return;  // disconnected continuation: dropped
    // Flavor sum of the loop-closing weight over the lanes of this configuration; the loop
    // factor sgn * w is already inside Md (the close's copy of the matrices).
    const double C = flavor_sum(close_value(csum), nfl, ci);
    if (SUBSETS && ones == 0u) {
        if (active && lam == 0) csub[(int64_t)B << cshift] = CLOW ? C : ldexp(C, __popc(B) - 1);
        if (dead) return;
    }
    if (ones) {
        const int k = __ffs(ones) - 1;
        const uint32_t bk = 1u << k;
        const uint32_t B1 = B | bk;
        const int hi1 = __popc(head_set(B1, A & ~B1) & (bk - 1u));
        const int ai1 = __popc(A & (bk - 1u));
        const uint32_t off1 = __ldg(tab.rank3 + code + c_p3[k]);
        T *tp = dst1 + (size_t)(off1 + (uint32_t)(hi1 * nA + ai1)) * kLanes + lane;
        double val = C;
        if (!CLOW && ell == 1 && shifts) val += sgn * 2.0 * sig;  // vertex 0 carries a shift point
        const T tv = narrow_to(T(0), val);
        if (CLOW) *tp = (k == 0 && lam == 0) ? T(0) : tv;        // k = 0: the head point is taken
        else if (k == 0) *tp += tv;                                // the extension into 0' wrote it
        else *tp = tv;
    } else if (active && lam == 0 && out) {
        const double c = CLOW ? C : ldexp(C, n - 1);
        out[cfg] = c;
        if (!isfinite(c)) atomicOr(status, kStatusNonFinite);
    }
}

// ------------------------------------------------------------------ double-float (df64) sweep
// The same row and mask steps with df64 states and matrices: every extension dot product and
// the loop-closing sum are Dot2 accumulations on the FP32 pipe (cos_df64.cuh); the flavor sum,
// the seeds and the sink stay in df64; only the sink's output is formed in FP64.

// Target slot of extension q for the row with head h, computed lane-parallel once per row
// (lane q holds the slot of the q-th extension; read back with one shuffle per push).
__device__ __forceinline__ uint32_t row_target_slot(const TgtInfo &ti, uint32_t hlow) {
    const uint32_t ai1 = ti.meta & 15u, nA1 = (ti.meta >> 4) & 15u;
    const uint32_t hi1 = (uint32_t)__popc((ti.meta >> 16) & hlow);
    return ti.off1 + hi1 * nA1 + ai1;
}

// The accumulator is stored as it stands (s, c): s + c is the value exactly, and an
// unnormalized pair only makes the next layer's dropped lo*lo term relative to the mass
// rather than to the state, which is the error model of this mode anyway.
__device__ __forceinline__ void push_target_df(df64 *__restrict__ dst1, uint32_t tslot, int q, const DotAcc &d,
                                               int lane) {
    const uint32_t slot = __shfl_sync(0xFFFFFFFFu, tslot, q);
    df64 v;
    v.hi = d.s;
    v.lo = d.c;
    dst1[(size_t)slot * kLanes + lane] = v;
}

template <int NV>
__device__ __forceinline__ void do_row_df(const df64 *__restrict__ src, df64 *__restrict__ dst1,
                                          const df64 *__restrict__ Ms, const df64 *__restrict__ Md,
                                          const TgtInfo &ti, int nJ, uint32_t J, uint32_t Vrow, uint32_t A,
                                          uint32_t off, int h, int hidx, int nA, int n, bool needclose, int lane,
                                          DotAcc &csum) {
    df64 o[NV];
    int vs[NV];
    const df64 *row = src + (size_t)(off + (uint32_t)(hidx * nA)) * kLanes + lane;
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
        for (int t = 0; t < NV; ++t) dot_add(csum, o[t], Md[vs[t] + h * kLanes]);
    }
    const uint32_t tslot = row_target_slot(ti, (1u << h) - 1u);
    uint32_t jj = J;
    int q = 0;
    for (; q + 1 < nJ; q += 2) {
        const int ja = __ffs(jj) - 1;
        jj &= jj - 1u;
        const int jb = __ffs(jj) - 1;
        jj &= jj - 1u;
        DotAcc da = dot_first(o[0], Ms[vs[0] + ja * kLanes]);
        DotAcc db = dot_first(o[0], Ms[vs[0] + jb * kLanes]);
#pragma unroll
        for (int t = 1; t < NV; ++t) {
            dot_add(da, o[t], Ms[vs[t] + ja * kLanes]);
            dot_add(db, o[t], Ms[vs[t] + jb * kLanes]);
        }
        push_target_df(dst1, tslot, q, da, lane);
        push_target_df(dst1, tslot, q + 1, db, lane);
    }
    if (q < nJ) {
        const int j = __ffs(jj) - 1;
        DotAcc d = dot_first(o[0], Ms[vs[0] + j * kLanes]);
#pragma unroll
        for (int t = 1; t < NV; ++t) dot_add(d, o[t], Ms[vs[t] + j * kLanes]);
        push_target_df(dst1, tslot, q, d, lane);
    }
}

__device__ __forceinline__ void row_dispatch_df(int nv, const df64 *src, df64 *dst1, const df64 *Ms, const df64 *Md,
                                                const TgtInfo &ti, int nJ, uint32_t J, uint32_t Vrow, uint32_t A,
                                                uint32_t off, int h, int hidx, int nA, int n, bool needclose,
                                                int lane, DotAcc &csum) {
#define COS_ROW_DF(K)                                                                                          \
    case K:                                                                                                    \
        do_row_df<K>(src, dst1, Ms, Md, ti, nJ, J, Vrow, A, off, h, hidx, nA, n, needclose, lane, csum);       \
        break;
    switch (nv) {
        COS_ROW_DF(1)
        COS_ROW_DF(2)
        COS_ROW_DF(3)
        COS_ROW_DF(4)
        COS_ROW_DF(5)
        COS_ROW_DF(6)
        COS_ROW_DF(7)
        COS_ROW_DF(8)
        COS_ROW_DF(9)
        COS_ROW_DF(10)
        COS_ROW_DF(11)
        COS_ROW_DF(12)
        default:
            break;
    }
#undef COS_ROW_DF
}

// One interaction mask of the df64 forward sweep (twin of fwd_mask).  seed0 = sgn 2 sigma as
// df64 (the shifted start at vertex 0, added at layer 1 when shifts are on).
template <bool SUBSETS = false>
__device__ __forceinline__ void fwd_mask_df(const OrderTab &tab, uint32_t mask_index, uint32_t next_index, int ell,
                                            int n, const df64 *src, df64 *dst1, const df64 *Ms, const df64 *Md,
                                            int lane, int ci, int nfl, df64 seed0, bool shifts, bool active, int lam,
                                            int cfg, double *out, int *status, int prefetch, double *csub = nullptr,
                                            int cshift = 0) {
    const uint32_t full = (1u << n) - 1u;
    const uint4 mk = __ldg(reinterpret_cast<const uint4 *>(tab.masks + mask_index));
    const uint32_t A = mk.x & 0xFFFFu, B = mk.x >> 16, code = mk.y, off = mk.z;
    const uint32_t ones = A & ~B;
    const uint32_t H = head_set(B, ones);
    const uint32_t J = full & ~B;
    const int nA = __popc(A);
    const bool dead = (ones == 0u) && (B != full);
    const bool needclose = !dead || SUBSETS;
    if (prefetch > 0 && next_index != 0xFFFFFFFFu) {
        const uint4 nk = __ldg(reinterpret_cast<const uint4 *>(tab.masks + next_index));
        const uint32_t nA_ = nk.x & 0xFFFFu, nB_ = nk.x >> 16;
        prefetch_block(reinterpret_cast<const double *>(src), nk.z,
                       (uint32_t)(__popc(head_set(nB_, nA_ & ~nB_)) * __popc(nA_)), lane, prefetch);
    }
    DotAcc csum = {0.0f, 0.0f};
    const TgtInfo ti = mask_targets(A, B, J, code, tab.rank3, lane);
    const int nJ = __popc(J);
    for (uint32_t hh = H; hh; hh &= hh - 1u) {
        const int h = __ffs(hh) - 1;
        const int hidx = __popc(H & ((1u << h) - 1u));
        const uint32_t Vrow = row_vmask(A, ones, h);
        row_dispatch_df(__popc(Vrow), src, dst1, Ms, Md, ti, nJ, J, Vrow, A, off, h, hidx, nA, n, needclose, lane,
                        csum);
    }
    if (!needclose) return;
    const df64 C = df64_flavor_sum(dot_value(csum), nfl, ci);
    if (SUBSETS && ones == 0u) {
        if (active && lam == 0) csub[(int64_t)B << cshift] = ldexp(df64_to_double(C), __popc(B) - 1);
        if (dead) return;
    }
    if (ones) {
        const int k = __ffs(ones) - 1;
        const uint32_t bk = 1u << k;
        const uint32_t B1 = B | bk;
        const int hi1 = __popc(head_set(B1, A & ~B1) & (bk - 1u));
        const int ai1 = __popc(A & (bk - 1u));
        const uint32_t off1 = __ldg(tab.rank3 + code + c_p3[k]);
        df64 *tp = dst1 + (size_t)(off1 + (uint32_t)(hi1 * nA + ai1)) * kLanes + lane;
        df64 val = C;
        if (ell == 1 && shifts) val = df64_add(val, seed0);   // vertex 0 carries a shift point
        if (k == 0) *tp = df64_add(*tp, val);                // the extension into 0' wrote it
        else *tp = val;
    } else if (active && lam == 0 && out) {
        const double c = ldexp(df64_to_double(C), n - 1);
        out[cfg] = c;
        if (!isfinite(c)) atomicOr(status, kStatusNonFinite);
    }
}

}  // namespace cosdp
