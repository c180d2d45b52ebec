// Double-float ("df64") arithmetic for the DP on the FP32 pipe.
//
// A value is an unevaluated sum hi + lo of two binary32 numbers, about 48 significant bits.
// Matrices, flavor sums and seeds are normalized (|lo| <= ulp(hi) / 2); DP states are stored
// as the dot-product accumulator leaves them (leading sum, error sum), whose sum is exact.
// On B300 the FP32 pipe retires 64 times as many lane operations per clock as the FP64 pipe,
// so a dot product kept in FP32 pairs costs less than one in FP64 while keeping a relative
// accuracy near 2^-47 per operation.  The building blocks are the classical
// error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2 4.2.2):  s = fl(a + b), e = (a + b) - s exactly, 6 additions;
//   TwoProd with FMA:                    p = fl(a b),  e = fma(a, b, -p) = a b - p exactly;
// and the compensated dot product of Ogita, Rump and Oishi ("Accurate sum and dot product",
// SIAM J. Sci. Comput. 26 (2005), algorithm Dot2), which sums the products' leading parts with
// TwoSum and collects every rounding error -- plus the cross terms hi*lo of the df64 inputs --
// in a second FP32 accumulator.  The (sum, error) pair is returned unrounded as a df64 value.
// The lo*lo cross term (relative size 2^-48) is dropped.
//
// Every operation uses the _rn intrinsics, which the compiler never contracts or reorders.
// Overflow and underflow follow binary32: the DP's states stay far inside its range for the
// orders this library accepts (|state| <= mass, products of at most 2n propagator entries).
#pragma once

#include <cuda_runtime.h>

namespace cosdp {

struct __align__(8) df64 {
    float hi, lo;
};

__device__ __forceinline__ float two_sum(float a, float b, float &e) {
    const float s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
    return s;
}

// Split of a binary64 value into hi + lo (hi = nearest float, lo = nearest float of the rest).
__device__ __forceinline__ df64 df64_from(double x) {
    df64 r;
    r.hi = __double2float_rn(x);
    r.lo = __double2float_rn(x - (double)r.hi);
    return r;
}

__device__ __forceinline__ double df64_to_double(df64 a) { return (double)a.hi + (double)a.lo; }

// a + b with a normalized result (sloppy addition: error <= 2^-45 (|a| + |b|)); the inputs
// may be unnormalized pairs.
__device__ __forceinline__ df64 df64_add(df64 a, df64 b) {
    float e;
    const float s = two_sum(a.hi, b.hi, e);
    const float t = __fadd_rn(__fadd_rn(a.lo, b.lo), e);
    df64 r;
    r.hi = two_sum(s, t, r.lo);
    return r;
}

// Compensated dot-product accumulator: value = s + c.
struct DotAcc {
    float s, c;
};

// First term x * y: the product's leading part and its exact error plus the cross terms.
__device__ __forceinline__ DotAcc dot_first(df64 x, df64 y) {
    DotAcc a;
    a.s = __fmul_rn(x.hi, y.hi);
    float c = __fmaf_rn(x.hi, y.hi, -a.s);
    c = __fmaf_rn(x.hi, y.lo, c);
    a.c = __fmaf_rn(x.lo, y.hi, c);
    return a;
}

// acc += x * y (Dot2 step on df64 operands): 1 multiply, 3 FMA, 8 additions.
__device__ __forceinline__ void dot_add(DotAcc &acc, df64 x, df64 y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float c = __fmaf_rn(x.hi, y.hi, -p);
    c = __fmaf_rn(x.hi, y.lo, c);
    c = __fmaf_rn(x.lo, y.hi, c);
    float e;
    acc.s = two_sum(acc.s, p, e);
    acc.c = __fadd_rn(acc.c, __fadd_rn(c, e));
}

// The accumulator as a normalized df64 value (TwoSum, valid under cancellation in s).
__device__ __forceinline__ df64 dot_value(DotAcc a) {
    df64 r;
    r.hi = two_sum(a.s, a.c, r.lo);
    return r;
}

// Sum of v over the nfl lanes of configuration ci, identical bits in every lane of the group
// (df64_add is commutative bit for bit: TwoSum's error term is exact, the lo additions commute).
__device__ __forceinline__ df64 df64_flavor_sum(df64 v, int nfl, int ci) {
    if (nfl == 1) return v;
    if ((nfl & (nfl - 1)) == 0) {
        for (int o = 1; o < nfl; o <<= 1) {
            df64 w;
            w.hi = __shfl_xor_sync(0xFFFFFFFFu, v.hi, o);
            w.lo = __shfl_xor_sync(0xFFFFFFFFu, v.lo, o);
            v = df64_add(v, w);
        }
        return v;
    }
    const int base = ci * nfl;
    df64 t;
    t.hi = __shfl_sync(0xFFFFFFFFu, v.hi, base & 31);
    t.lo = __shfl_sync(0xFFFFFFFFu, v.lo, base & 31);
    for (int g = 1; g < nfl; ++g) {
        df64 w;
        w.hi = __shfl_sync(0xFFFFFFFFu, v.hi, (base + g) & 31);
        w.lo = __shfl_sync(0xFFFFFFFFu, v.lo, (base + g) & 31);
        t = df64_add(t, w);
    }
    return t;
}

}  // namespace cosdp
