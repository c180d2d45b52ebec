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

// ------------------------------------------------------------------ two configurations per instruction
// The kernels that carry several configurations per lane run the same operation sequence for
// each of them, so the FP32 arithmetic is issued in packed pairs: sm_100-family packed FP32
// (.f32x2) performs two round-to-nearest operations in one issue slot, each bit for bit the
// scalar operation.  A float2 holds one value of configuration pair (x, y).  Subtraction has no
// CUDA intrinsic; it is the PTX sub.rn.f32x2 instruction.

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long r;
    const unsigned long long x = (unsigned long long)__float_as_uint(a.x) | ((unsigned long long)__float_as_uint(a.y) << 32);
    const unsigned long long y = (unsigned long long)__float_as_uint(b.x) | ((unsigned long long)__float_as_uint(b.y) << 32);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
    return make_float2(__uint_as_float((unsigned)r), __uint_as_float((unsigned)(r >> 32)));
}
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// TwoSum of each component (as two_sum).
__device__ __forceinline__ float2 two_sum2(float2 a, float2 b, float2 &e) {
    const float2 s = add2(a, b);
    const float2 z = sub2(s, a);
    e = add2(sub2(a, sub2(s, z)), sub2(b, z));
    return s;
}

// Two df64 values (configurations x and y) of one lane, stored as (hi pair, lo pair) so that each
// pair is one packed-FP32 operand.
struct __align__(16) df64x2 {
    float2 hi, lo;
};
__device__ __forceinline__ df64 dfx(const df64x2 &v) { return df64{v.hi.x, v.lo.x}; }
__device__ __forceinline__ df64 dfy(const df64x2 &v) { return df64{v.hi.y, v.lo.y}; }
__device__ __forceinline__ df64x2 dfpair(df64 x, df64 y) {
    df64x2 r;
    r.hi = make_float2(x.hi, y.hi);
    r.lo = make_float2(x.lo, y.lo);
    return r;
}

// Compensated dot-product accumulators of two configurations: value = s + c per component.
struct DotAcc2 {
    float2 s, c;
};

// acc += x * y per component, x and y given as (hi, lo) pairs of float2 (dot_add's steps).
__device__ __forceinline__ void dot_add2(DotAcc2 &acc, float2 xhi, float2 xlo, float2 yhi, float2 ylo) {
    const float2 p = mul2(xhi, yhi);
    float2 c = fma2(xhi, yhi, neg2(p));
    c = fma2(xhi, ylo, c);
    c = fma2(xlo, yhi, c);
    float2 e;
    acc.s = two_sum2(acc.s, p, e);
    acc.c = add2(acc.c, add2(c, e));
}

// First term (dot_first's steps).
__device__ __forceinline__ DotAcc2 dot_first2(float2 xhi, float2 xlo, float2 yhi, float2 ylo) {
    DotAcc2 a;
    a.s = mul2(xhi, yhi);
    float2 c = fma2(xhi, yhi, neg2(a.s));
    c = fma2(xhi, ylo, c);
    a.c = fma2(xlo, yhi, c);
    return a;
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
