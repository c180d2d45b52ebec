// Mixed-precision DP with two configurations per lane.
//
// In the mixed mode (FP32 extension, FP64 close) the FP32 multiply-adds are cheap and the
// warp-uniform index work of a mask -- target offsets, endpoint slots, shuffles, stores --
// dominates the issue slots.  Here every lane carries the same flavor of two configurations
// (the .x and .y components of a float2 state), so each index computation, shared-memory
// address and branch serves two configurations: a batch holds 2 x floor(32 / n_flavors)
// configurations.  The arithmetic per configuration is that of dp_forward_kernel<float>:
// FP32 extension states and accumulation, the compensated FP32-pair close (widened and added
// in FP64 once per mask), seeds rounded to FP32, flavor sums in FP64 (one butterfly per
// component, identical bits in every lane of a configuration), and the sink in FP64.  Layout
// (P configurations per lane): states [slot][lane] as P floats, extension matrices
// [v][j][lane] as P floats, close matrices (times sgn w) as P FP32 pairs.
//
// The double-float mode (FP32 pairs) is issue-bound for the same reason and gets the same
// treatment: df64x2 states (two df64 values, 16 bytes per lane), compensated accumulation
// per component, df64 flavor sums and seeds, the sink in FP64.
#include <algorithm>
#include <cstring>

#include "cos_dp_device.cuh"

namespace cosdp {

namespace {

// P floats of one lane (one per configuration), aligned for single vector accesses; the close
// matrices as P FP32 pairs hi + lo (the compensated close of cos_dp_device.cuh).
template <int P>
struct __align__(4 * P) FV {
    float v[P];
};
template <int P>
struct __align__(16) CV {
    float hi[P], lo[P];
};

// Configurations per lane of the mixed kernel.
constexpr int kMixedWidth = 4;

// 128-bit shared-memory load at a byte address of the shared window (the row steps keep 32-bit
// addresses per state, so an extension's matrix load costs one add).
__device__ __forceinline__ float4 lds4(uint32_t addr) {
    float4 r;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "r"(addr));
    return r;
}

// Pulls `nslots` state slots from slot `off` on (16 bytes per lane: four 128-byte lines a slot)
// into L1, one line per lane and instruction.  Used one row ahead (prefetch mode 3): the loads of
// a row are issued together and the warp then computes with nothing in flight, so a warp would
// otherwise keep about one row of DRAM reads outstanding.
__device__ __forceinline__ void prefetch_rows_l1(const void *src, uint32_t off, uint32_t nslots, int lane) {
    const char *base = reinterpret_cast<const char *>(src) + (size_t)off * (kLanes * 16);
    for (uint32_t l = (uint32_t)lane; l < 4u * nslots; l += kLanes)
        asm volatile("prefetch.global.L1 [%0];" ::"l"(base + (size_t)l * 128));
}

// One row (mu, h) of the mixed mode, four configurations per lane (float4 states: packed pairs
// (x, y) and (z, w)).  ms / md: shared byte addresses of Ms[0][0][0] and Md[0][0][0]; an entry
// [v][j] of lane l sits at ((v n + j) 32 + l) times its size (16 bytes, 32 for Md).  The row's
// target slots are formed lane-parallel once (lane q: extension q) and read with one shuffle per
// push.
// CONT: the row's second part (rows longer than kRowStates run in two parts): the extension dot
// products continue from the values the first part stored in the target slots (the same FMA
// chain, so the same bits as one pass).
template <int NV, bool CONT = false>
__device__ __forceinline__ void do_row_pair(const FV<4> *__restrict__ src, FV<4> *__restrict__ dst1, uint32_t ms,
                                            uint32_t md, const TgtInfo &ti, int nJ, uint32_t J, uint32_t Vrow,
                                            uint32_t A, uint32_t off, int h, int hidx, int nA, int n, bool needclose,
                                            int lane, DotAcc2 (&csum)[2]) {
    float4 o[NV];
    uint32_t ma[NV];   // byte address of Ms[v_t][0] for this lane
    const float4 *row = reinterpret_cast<const float4 *>(src) + (size_t)(off + (uint32_t)(hidx * nA)) * kLanes + lane;
    uint32_t vv = Vrow;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        const int v = __ffs(vv) - 1;
        vv &= vv - 1u;
        o[t] = row[__popc(A & ((1u << v) - 1u)) * kLanes];
        ma[t] = ms + (uint32_t)((v * n * kLanes + lane) * 16);
    }
    if (needclose) {
        // Md[v][h] = 2 (Ms[v][0] - ms) + md + h 32 32 bytes
        const uint32_t dh = md + (uint32_t)(h * kLanes * 32) - 2u * ms;
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            const uint32_t a = 2u * ma[t] + dh;
            const float4 hi = lds4(a), lo = lds4(a + 16u);
            close_add2(csum[0], make_float2(o[t].x, o[t].y), make_float2(hi.x, hi.y), make_float2(lo.x, lo.y));
            close_add2(csum[1], make_float2(o[t].z, o[t].w), make_float2(hi.z, hi.w), make_float2(lo.z, lo.w));
        }
    }
    const uint32_t tslot = row_target_slot(ti, (1u << h) - 1u);
    float4 *dl = reinterpret_cast<float4 *>(dst1) + lane;
    uint32_t jj = J;
    int q = 0;
    for (; q + 1 < nJ; q += 2) {
        const uint32_t ja = (uint32_t)(__ffs(jj) - 1) * (kLanes * 16);
        jj &= jj - 1u;
        const uint32_t jb = (uint32_t)(__ffs(jj) - 1) * (kLanes * 16);
        jj &= jj - 1u;
        const uint32_t sa = __shfl_sync(0xFFFFFFFFu, tslot, q), sb = __shfl_sync(0xFFFFFFFFu, tslot, q + 1);
        float2 a0 = make_float2(0.0f, 0.0f), a1 = a0, b0 = a0, b1 = a0;
        if constexpr (CONT) {
            const float4 pa = dl[(size_t)sa * kLanes], pb = dl[(size_t)sb * kLanes];
            a0 = make_float2(pa.x, pa.y);
            a1 = make_float2(pa.z, pa.w);
            b0 = make_float2(pb.x, pb.y);
            b1 = make_float2(pb.z, pb.w);
        }
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            const float4 ma_ = lds4(ma[t] + ja), mb_ = lds4(ma[t] + jb);
            const float2 o0 = make_float2(o[t].x, o[t].y), o1 = make_float2(o[t].z, o[t].w);
            a0 = fma2(o0, make_float2(ma_.x, ma_.y), a0);
            a1 = fma2(o1, make_float2(ma_.z, ma_.w), a1);
            b0 = fma2(o0, make_float2(mb_.x, mb_.y), b0);
            b1 = fma2(o1, make_float2(mb_.z, mb_.w), b1);
        }
        dl[(size_t)sa * kLanes] = make_float4(a0.x, a0.y, a1.x, a1.y);
        dl[(size_t)sb * kLanes] = make_float4(b0.x, b0.y, b1.x, b1.y);
    }
    if (q < nJ) {
        const uint32_t jo = (uint32_t)(__ffs(jj) - 1) * (kLanes * 16);
        const uint32_t sq = __shfl_sync(0xFFFFFFFFu, tslot, q);
        float2 d0 = make_float2(0.0f, 0.0f), d1 = d0;
        if constexpr (CONT) {
            const float4 pd = dl[(size_t)sq * kLanes];
            d0 = make_float2(pd.x, pd.y);
            d1 = make_float2(pd.z, pd.w);
        }
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            const float4 m = lds4(ma[t] + jo);
            d0 = fma2(make_float2(o[t].x, o[t].y), make_float2(m.x, m.y), d0);
            d1 = fma2(make_float2(o[t].z, o[t].w), make_float2(m.z, m.w), d1);
        }
        dl[(size_t)sq * kLanes] = make_float4(d0.x, d0.y, d1.x, d1.y);
    }
}

// Longest row part run in one pass (the states of a part are held in registers; longer rows run
// in two parts, the second continuing the first's dot products).
constexpr int kRowStates = 6;

__device__ __forceinline__ void row_dispatch_pair(int nv, const FV<4> *src, FV<4> *dst1, uint32_t ms, uint32_t md,
                                                  const TgtInfo &ti, int nJ, uint32_t J, uint32_t Vrow, uint32_t A,
                                                  uint32_t off, int h, int hidx, int nA, int n, bool needclose,
                                                  int lane, DotAcc2 (&csum)[2]) {
#define COS_ROW_P(K, C, V)                                                                                     \
    case K:                                                                                                    \
        do_row_pair<K, C>(src, dst1, ms, md, ti, nJ, J, V, A, off, h, hidx, nA, n, needclose, lane, csum);     \
        break;
    uint32_t V2 = 0u;
    if (nv > kRowStates) {   // the first kRowStates endpoints, then the rest
        const uint32_t cut = 1u << (__fns(Vrow, 0, kRowStates + 1));
        V2 = Vrow & ~(cut - 1u);
        Vrow &= cut - 1u;
        nv = kRowStates;
    }
    switch (nv) {
        COS_ROW_P(1, false, Vrow)
        COS_ROW_P(2, false, Vrow)
        COS_ROW_P(3, false, Vrow)
        COS_ROW_P(4, false, Vrow)
        COS_ROW_P(5, false, Vrow)
        COS_ROW_P(6, false, Vrow)
        default:
            break;
    }
    if (V2) {
        switch (__popc(V2)) {
            COS_ROW_P(1, true, V2)
            COS_ROW_P(2, true, V2)
            COS_ROW_P(3, true, V2)
            COS_ROW_P(4, true, V2)
            COS_ROW_P(5, true, V2)
            COS_ROW_P(6, true, V2)
            default:
                break;
        }
    }
#undef COS_ROW_P
}

// One interaction mask for the P configurations of every lane (twin of fwd_mask<float>;
// CLOW: determinant weights without cycle factors, as there).
template <int P, bool CLOW>
__device__ __forceinline__ void fwd_mask_pair(const OrderTab &tab, uint32_t mask_index, uint32_t next_index, int ell,
                                              int n, const FV<P> *src, FV<P> *dst1, const FV<P> *Ms,
                                              const CV<P> *Md, int lane, int ci, int nfl, double sgn, double sig,
                                              bool shifts, const bool act[P], const int cfg[P], int lam, double *out,
                                              int *status, int prefetch) {
    const uint32_t full = (1u << n) - 1u;
    const uint4 mk = __ldg(reinterpret_cast<const uint4 *>(tab.masks + mask_index));
    const uint32_t A = mk.x & 0xFFFFu, B = mk.x >> 16, code = mk.y, off = mk.z;
    const uint32_t ones = A & ~B;
    const uint32_t H = head_set(B, ones);
    const uint32_t J = full & ~B & (CLOW ? ~(ones & 1u) : 0xFFFFFFFFu);
    const int nA = __popc(A);
    const bool needclose = (ones != 0u) || (B == full);
    if ((prefetch == 1 || prefetch == 2 || prefetch == 4) && next_index != 0xFFFFFFFFu) {
        // P * 4-byte states: P / 2 rows of 256 bytes per state slot
        const uint4 nk = __ldg(reinterpret_cast<const uint4 *>(tab.masks + next_index));
        const uint32_t nA_ = nk.x & 0xFFFFu, nB_ = nk.x >> 16;
        const uint32_t ns = (uint32_t)(__popc(head_set(nB_, nA_ & ~nB_)) * __popc(nA_));
        prefetch_block(reinterpret_cast<const double *>(src), (uint32_t)(P / 2) * nk.z, (uint32_t)(P / 2) * ns, lane,
                       prefetch == 4 ? 1 : prefetch);
    }
    DotAcc2 csum[P / 2];
#pragma unroll
    for (int k = 0; k < P / 2; ++k) csum[k].s = csum[k].c = make_float2(0.0f, 0.0f);
    const TgtInfo ti = mask_targets(A, B, J, code, tab.rank3, lane);
    const int nJ = __popc(J);
    for (uint32_t hh = H; hh; hh &= hh - 1u) {
        const int h = __ffs(hh) - 1;
        const int hidx = __popc(H & ((1u << h) - 1u));
        const uint32_t Vrow = row_vmask(A, ones, h);
        if (prefetch >= 3) {   // the next row of this mask, else the first row of the warp's next mask
            if (hh & (hh - 1u)) {
                prefetch_rows_l1(src, off + (uint32_t)((hidx + 1) * nA), (uint32_t)nA, lane);
            } else if (next_index != 0xFFFFFFFFu) {
                const uint4 nk = __ldg(reinterpret_cast<const uint4 *>(tab.masks + next_index));
                prefetch_rows_l1(src, nk.z, (uint32_t)__popc(nk.x & 0xFFFFu), lane);
            }
        }
        row_dispatch_pair(__popc(Vrow), src, dst1, (uint32_t)__cvta_generic_to_shared(Ms),
                          (uint32_t)__cvta_generic_to_shared(Md), ti, nJ, J, Vrow, A, off, h, hidx, nA, n, needclose,
                          lane, csum);
    }
    if (!needclose) return;   // no half-visited vertex and not full: disconnected, dropped
    double C[P];
#pragma unroll
    for (int c = 0; c < P; ++c) {
        const DotAcc2 &q = csum[c / 2];
        const DotAcc acc = (c & 1) ? DotAcc{q.s.y, q.c.y} : DotAcc{q.s.x, q.c.x};
        C[c] = flavor_sum(close_value(acc), nfl, ci);
    }
    if (ones) {
        const int k = __ffs(ones) - 1;
        const uint32_t bk = 1u << k;
        const uint32_t B1 = B | bk;
        const int hi1 = __popc(head_set(B1, A & ~B1) & (bk - 1u));
        const int ai1 = __popc(A & (bk - 1u));
        const uint32_t off1 = __ldg(tab.rank3 + code + c_p3[k]);
        FV<P> *tp = dst1 + (size_t)(off1 + (uint32_t)(hi1 * nA + ai1)) * kLanes + lane;
        FV<P> tv;
#pragma unroll
        for (int c = 0; c < P; ++c) {
            double v = C[c];
            if (!CLOW && ell == 1 && shifts) v += sgn * 2.0 * sig;   // vertex 0 carries a shift point
            tv.v[c] = (CLOW && k == 0 && lam == 0) ? 0.0f : narrow_to(0.0f, v);
        }
        if (!CLOW && k == 0) {                              // the extension into 0' wrote it
            FV<P> cur = *tp;
#pragma unroll
            for (int c = 0; c < P; ++c) cur.v[c] += tv.v[c];
            *tp = cur;
        } else {
            *tp = tv;
        }
    } else if (lam == 0 && out) {
#pragma unroll
        for (int c = 0; c < P; ++c)
            if (act[c]) {
                const double r = CLOW ? C[c] : ldexp(C[c], n - 1);
                out[cfg[c]] = r;
                if (!isfinite(r)) atomicOr(status, kStatusNonFinite);
            }
    }
}

// ---------------------------------------------------------------- double-float, two per lane

// df64x2 (two configurations' df64 values of a lane) and its accessors: cos_df64.cuh.

// The accumulators are stored as they stand (sum, error) for both configurations.
__device__ __forceinline__ void push_target_dfp(df64x2 *__restrict__ dst1, uint32_t tslot, int q, const DotAcc2 &d,
                                                int lane) {
    const uint32_t slot = __shfl_sync(0xFFFFFFFFu, tslot, q);
    df64x2 v;
    v.hi = d.s;
    v.lo = d.c;
    dst1[(size_t)slot * kLanes + lane] = v;
}

// One row of the double-float mode.  ms / md: shared byte addresses of Ms and Md (16-byte
// entries [v][j][lane], as in do_row_pair).
template <int NV>
__device__ __forceinline__ void do_row_dfp(const df64x2 *__restrict__ src, df64x2 *__restrict__ dst1, uint32_t ms,
                                           uint32_t md, const TgtInfo &ti, int nJ, uint32_t J, uint32_t Vrow,
                                           uint32_t A, uint32_t off, int h, int hidx, int nA, int n, bool needclose,
                                           int lane, DotAcc2 &cc) {
    df64x2 o[NV];
    uint32_t ma[NV];   // byte offset of entry [v_t][0] of this lane
    const df64x2 *row = src + (size_t)(off + (uint32_t)(hidx * nA)) * kLanes + lane;
    uint32_t vv = Vrow;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        const int v = __ffs(vv) - 1;
        vv &= vv - 1u;
        o[t] = row[__popc(A & ((1u << v) - 1u)) * kLanes];
        ma[t] = (uint32_t)((v * n * kLanes + lane) * 16);
    }
    if (needclose) {
        const uint32_t dh = md + (uint32_t)(h * kLanes * 16);
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            const float4 m = lds4(ma[t] + dh);
            dot_add2(cc, o[t].hi, o[t].lo, make_float2(m.x, m.y), make_float2(m.z, m.w));
        }
    }
#pragma unroll
    for (int t = 0; t < NV; ++t) ma[t] += ms;
    const uint32_t tslot = row_target_slot(ti, (1u << h) - 1u);
    uint32_t jj = J;
    int q = 0;
    for (; q + 1 < nJ; q += 2) {
        const uint32_t ja = (uint32_t)(__ffs(jj) - 1) * (kLanes * 16);
        jj &= jj - 1u;
        const uint32_t jb = (uint32_t)(__ffs(jj) - 1) * (kLanes * 16);
        jj &= jj - 1u;
        const float4 ma0 = lds4(ma[0] + ja), mb0 = lds4(ma[0] + jb);
        DotAcc2 da = dot_first2(o[0].hi, o[0].lo, make_float2(ma0.x, ma0.y), make_float2(ma0.z, ma0.w));
        DotAcc2 db = dot_first2(o[0].hi, o[0].lo, make_float2(mb0.x, mb0.y), make_float2(mb0.z, mb0.w));
#pragma unroll
        for (int t = 1; t < NV; ++t) {
            const float4 a_ = lds4(ma[t] + ja), b_ = lds4(ma[t] + jb);
            dot_add2(da, o[t].hi, o[t].lo, make_float2(a_.x, a_.y), make_float2(a_.z, a_.w));
            dot_add2(db, o[t].hi, o[t].lo, make_float2(b_.x, b_.y), make_float2(b_.z, b_.w));
        }
        push_target_dfp(dst1, tslot, q, da, lane);
        push_target_dfp(dst1, tslot, q + 1, db, lane);
    }
    if (q < nJ) {
        const uint32_t jo = (uint32_t)(__ffs(jj) - 1) * (kLanes * 16);
        const float4 m0 = lds4(ma[0] + jo);
        DotAcc2 d = dot_first2(o[0].hi, o[0].lo, make_float2(m0.x, m0.y), make_float2(m0.z, m0.w));
#pragma unroll
        for (int t = 1; t < NV; ++t) {
            const float4 m = lds4(ma[t] + jo);
            dot_add2(d, o[t].hi, o[t].lo, make_float2(m.x, m.y), make_float2(m.z, m.w));
        }
        push_target_dfp(dst1, tslot, q, d, lane);
    }
}

__device__ __forceinline__ void row_dispatch_dfp(int nv, const df64x2 *src, df64x2 *dst1, uint32_t Ms, uint32_t Md,
                                                 const TgtInfo &ti, int nJ, uint32_t J,
                                                 uint32_t Vrow, uint32_t A, uint32_t off, int h, int hidx, int nA,
                                                 int n, bool needclose, int lane, DotAcc2 &cc) {
#define COS_ROW_DP(K)                                                                                          \
    case K:                                                                                                    \
        do_row_dfp<K>(src, dst1, Ms, Md, ti, nJ, J, Vrow, A, off, h, hidx, nA, n, needclose, lane, cc);        \
        break;
    switch (nv) {
        COS_ROW_DP(1)
        COS_ROW_DP(2)
        COS_ROW_DP(3)
        COS_ROW_DP(4)
        COS_ROW_DP(5)
        COS_ROW_DP(6)
        COS_ROW_DP(7)
        COS_ROW_DP(8)
        COS_ROW_DP(9)
        COS_ROW_DP(10)
        COS_ROW_DP(11)
        COS_ROW_DP(12)
        default:
            break;
    }
#undef COS_ROW_DP
}

template <bool CLOW>
__device__ __forceinline__ void fwd_mask_dfp(const OrderTab &tab, uint32_t mask_index, uint32_t next_index, int ell,
                                             int n, const df64x2 *src, df64x2 *dst1, const df64x2 *Ms,
                                             const df64x2 *Md, int lane, int ci, int nfl, df64 seed0, bool shifts,
                                             bool act_x, bool act_y, int lam, int cfg_x, int cfg_y, double *out,
                                             int *status, int prefetch) {
    const uint32_t full = (1u << n) - 1u;
    const uint4 mk = __ldg(reinterpret_cast<const uint4 *>(tab.masks + mask_index));
    const uint32_t A = mk.x & 0xFFFFu, B = mk.x >> 16, code = mk.y, off = mk.z;
    const uint32_t ones = A & ~B;
    const uint32_t H = head_set(B, ones);
    const uint32_t J = full & ~B & (CLOW ? ~(ones & 1u) : 0xFFFFFFFFu);
    const int nA = __popc(A);
    const bool needclose = (ones != 0u) || (B == full);
    if ((prefetch == 1 || prefetch == 2 || prefetch == 4) && next_index != 0xFFFFFFFFu) {
        // 16-byte states: two 256-byte lines per warp row, fetched as two double-sized rows
        const uint4 nk = __ldg(reinterpret_cast<const uint4 *>(tab.masks + next_index));
        const uint32_t nA_ = nk.x & 0xFFFFu, nB_ = nk.x >> 16;
        const uint32_t ns = (uint32_t)(__popc(head_set(nB_, nA_ & ~nB_)) * __popc(nA_));
        prefetch_block(reinterpret_cast<const double *>(src), 2 * nk.z, 2 * ns, lane, prefetch == 4 ? 1 : prefetch);
    }
    DotAcc2 cc;
    cc.s = cc.c = make_float2(0.0f, 0.0f);
    const TgtInfo ti = mask_targets(A, B, J, code, tab.rank3, lane);
    const int nJ = __popc(J);
    for (uint32_t hh = H; hh; hh &= hh - 1u) {
        const int h = __ffs(hh) - 1;
        const int hidx = __popc(H & ((1u << h) - 1u));
        const uint32_t Vrow = row_vmask(A, ones, h);
        if (prefetch >= 3) {   // the next row of this mask, else the first row of the warp's next mask
            if (hh & (hh - 1u)) {
                prefetch_rows_l1(src, off + (uint32_t)((hidx + 1) * nA), (uint32_t)nA, lane);
            } else if (next_index != 0xFFFFFFFFu) {
                const uint4 nk = __ldg(reinterpret_cast<const uint4 *>(tab.masks + next_index));
                prefetch_rows_l1(src, nk.z, (uint32_t)__popc(nk.x & 0xFFFFu), lane);
            }
        }
        row_dispatch_dfp(__popc(Vrow), src, dst1, (uint32_t)__cvta_generic_to_shared(Ms),
                         (uint32_t)__cvta_generic_to_shared(Md), ti, nJ, J, Vrow, A, off, h, hidx, nA, n, needclose,
                         lane, cc);
    }
    if (!needclose) return;
    const df64 Cx = df64_flavor_sum(dot_value(DotAcc{cc.s.x, cc.c.x}), nfl, ci);
    const df64 Cy = df64_flavor_sum(dot_value(DotAcc{cc.s.y, cc.c.y}), nfl, ci);
    if (ones) {
        const int k = __ffs(ones) - 1;
        const uint32_t bk = 1u << k;
        const uint32_t B1 = B | bk;
        const int hi1 = __popc(head_set(B1, A & ~B1) & (bk - 1u));
        const int ai1 = __popc(A & (bk - 1u));
        const uint32_t off1 = __ldg(tab.rank3 + code + c_p3[k]);
        df64x2 *tp = dst1 + (size_t)(off1 + (uint32_t)(hi1 * nA + ai1)) * kLanes + lane;
        df64 vx = Cx, vy = Cy;
        if (!CLOW && ell == 1 && shifts) {   // vertex 0 carries a shift point
            vx = df64_add(vx, seed0);
            vy = df64_add(vy, seed0);
        }
        if (CLOW && k == 0 && lam == 0) vx = vy = df64{0.0f, 0.0f};   // block 1 only
        if (!CLOW && k == 0) {               // the extension into 0' wrote it
            const df64x2 cur = *tp;
            *tp = dfpair(df64_add(dfx(cur), vx), df64_add(dfy(cur), vy));
        } else {
            *tp = dfpair(vx, vy);
        }
    } else if (lam == 0 && out) {
        if (act_x) {
            const double c = CLOW ? df64_to_double(Cx) : ldexp(df64_to_double(Cx), n - 1);
            out[cfg_x] = c;
            if (!isfinite(c)) atomicOr(status, kStatusNonFinite);
        }
        if (act_y) {
            const double c = CLOW ? df64_to_double(Cy) : ldexp(df64_to_double(Cy), n - 1);
            out[cfg_y] = c;
            if (!isfinite(c)) atomicOr(status, kStatusNonFinite);
        }
    }
}

}  // namespace

// MAXT = 256 (two CTAs of up to 8 warps, <= 128 registers), 384 (two CTAs of up to 12 warps,
// <= 85), 512 (one CTA of up to 16 warps, <= 128) or 640 (one CTA of up to 20 warps, <= 102).
template <int MAXT, bool CLOW>
__global__ void __launch_bounds__(MAXT, MAXT <= 384 ? 2 : 1) dp_pair_dfp_kernel(const __grid_constant__ DpArgs a);

template <int P, int MAXT, bool CLOW>
__global__ void __launch_bounds__(MAXT, MAXT <= 384 ? 2 : 1) dp_pair_kernel(const __grid_constant__ DpArgs a) {
    extern __shared__ __align__(16) unsigned char smem_p[];
    __shared__ int s_batch;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int nsm = a.smem_n * a.smem_n * kLanes;
    FV<P> *Ms = reinterpret_cast<FV<P> *>(smem_p);
    CV<P> *Md = reinterpret_cast<CV<P> *>(smem_p + (((size_t)nsm * sizeof(FV<P>) + 15) & ~size_t(15)));
    FV<P> *ring = reinterpret_cast<FV<P> *>(a.scratch) + (size_t)blockIdx.x * a.nslots * a.slot_elems;
    const int nfl = a.nf_lanes;
    const int lam = lane % nfl;
    const int ci = lane / nfl;
    const int cpl = kLanes / nfl;   // configurations per component
    const double sgn = a.absmode ? 1.0 : -1.0;
    const double sig = a.absmode ? fabs(a.sigma[lam]) : a.sigma[lam];
    const bool shifts = a.shifts != 0;
    const int nbatch = *a.n_batches;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_batch = atomicAdd(a.queue, 1);
        __syncthreads();
        const int b = s_batch;
        if (b >= nbatch) break;
        const int4 bd = a.batches[b];
        const int n = bd.x;
        const OrderTab &tab = a.tabs[n];
        const bool lane_ok = ci * nfl + nfl <= kLanes;
        bool act[P];
        int cfg[P];
        const double *Mp[P];
#pragma unroll
        for (int c = 0; c < P; ++c) {
            act[c] = lane_ok && (ci + c * cpl < bd.z);
            cfg[c] = act[c] ? a.batch_list[bd.y + c * cpl + ci] : -1;
            Mp[c] = act[c] ? a.M + (a.moff ? a.moff[cfg[c]] : (int64_t)cfg[c] * a.mstride) + (size_t)lam * n * n
                           : nullptr;
        }
        const double cfac = sgn * a.loop_weight;
        const double dshift = sgn * sig;
        for (int e = warp; e < n * n; e += nwarps) {
            const int v = e / n, j = e % n;
            const bool sh = v == j && (CLOW || (j != 0 && shifts));
            FV<P> m;
            CV<P> d;
#pragma unroll
            for (int c = 0; c < P; ++c) {
                double val = act[c] ? Mp[c][e] : 0.0;
                if (a.absmode) val = fabs(val);
                m.v[c] = (float)(sh ? val + dshift : val);
                // CLOW: shifted diagonal in the close too
                const df64 md = df64_from(cfac * ((CLOW && sh) ? val + dshift : val));
                d.hi[c] = md.hi;
                d.lo[c] = md.lo;
            }
            Ms[e * kLanes + lane] = m;
            Md[e * kLanes + lane] = d;
        }
        if (warp == 0) {
            FV<P> one;
#pragma unroll
            for (int c = 0; c < P; ++c) one.v[c] = (CLOW && lam != 0) ? 0.0f : 1.0f;
            ring[(1 % a.nslots) * a.slot_elems + lane] = one;
        }
        __syncthreads();
        for (int ell = 1; ell <= 2 * n; ++ell) {
            const FV<P> *src = ring + (size_t)(ell % a.nslots) * a.slot_elems;
            FV<P> *dst1 = ring + (size_t)((ell + 1) % a.nslots) * a.slot_elems;
            const uint32_t first = tab.layer_first[ell];
            const uint32_t cnt = tab.layer_count[ell];
            for (uint32_t mi = warp; mi < cnt; mi += nwarps)
                fwd_mask_pair<P, CLOW>(tab, first + mi, mi + nwarps < cnt ? first + mi + nwarps : 0xFFFFFFFFu, ell, n, src,
                                 dst1, Ms, Md, lane, ci, nfl, sgn, sig, shifts, act, cfg, lam, a.out, a.status,
                                 a.prefetch);
            __syncthreads();
        }
    }
}

template <int MAXT, bool CLOW>
__global__ void __launch_bounds__(MAXT, MAXT <= 384 ? 2 : 1) dp_pair_dfp_kernel(const __grid_constant__ DpArgs a) {
    extern __shared__ __align__(16) unsigned char smem_q[];
    __shared__ int s_batch;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int nsm = a.smem_n * a.smem_n * kLanes;
    df64x2 *Ms = reinterpret_cast<df64x2 *>(smem_q);
    df64x2 *Md = Ms + nsm;
    df64x2 *ring = reinterpret_cast<df64x2 *>(a.scratch) + (size_t)blockIdx.x * a.nslots * a.slot_elems;
    const int nfl = a.nf_lanes;
    const int lam = lane % nfl;
    const int ci = lane / nfl;
    const int cpl = kLanes / nfl;
    const double sgn = a.absmode ? 1.0 : -1.0;
    const double sig = a.absmode ? fabs(a.sigma[lam]) : a.sigma[lam];
    const bool shifts = a.shifts != 0;
    const df64 seed0 = df64_from(sgn * 2.0 * sig);
    const int nbatch = *a.n_batches;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_batch = atomicAdd(a.queue, 1);
        __syncthreads();
        const int b = s_batch;
        if (b >= nbatch) break;
        const int4 bd = a.batches[b];
        const int n = bd.x;
        const OrderTab &tab = a.tabs[n];
        const bool lane_ok = ci * nfl + nfl <= kLanes;
        const bool act_x = lane_ok && (ci < bd.z);
        const bool act_y = lane_ok && (ci + cpl < bd.z);
        const int cfg_x = act_x ? a.batch_list[bd.y + ci] : -1;
        const int cfg_y = act_y ? a.batch_list[bd.y + cpl + ci] : -1;
        const double *Mx = act_x ? a.M + (a.moff ? a.moff[cfg_x] : (int64_t)cfg_x * a.mstride) + (size_t)lam * n * n
                                 : nullptr;
        const double *My = act_y ? a.M + (a.moff ? a.moff[cfg_y] : (int64_t)cfg_y * a.mstride) + (size_t)lam * n * n
                                 : nullptr;
        const double cfac = sgn * a.loop_weight;
        const double dshift = sgn * sig;
        for (int e = warp; e < n * n; e += nwarps) {
            double vx = act_x ? Mx[e] : 0.0, vy = act_y ? My[e] : 0.0;
            if (a.absmode) {
                vx = fabs(vx);
                vy = fabs(vy);
            }
            const int v = e / n, j = e % n;
            const bool sh = v == j && (CLOW || (j != 0 && shifts));
            Ms[e * kLanes + lane] = dfpair(df64_from(sh ? vx + dshift : vx), df64_from(sh ? vy + dshift : vy));
            // CLOW: shifted diagonal in the close too
            Md[e * kLanes + lane] = dfpair(df64_from(cfac * ((CLOW && sh) ? vx + dshift : vx)),
                                           df64_from(cfac * ((CLOW && sh) ? vy + dshift : vy)));
        }
        if (warp == 0) {
            const float s0 = (CLOW && lam != 0) ? 0.0f : 1.0f;
            ring[(1 % a.nslots) * a.slot_elems + lane] = dfpair(df64{s0, 0.0f}, df64{s0, 0.0f});
        }
        __syncthreads();
        for (int ell = 1; ell <= 2 * n; ++ell) {
            const df64x2 *src = ring + (size_t)(ell % a.nslots) * a.slot_elems;
            df64x2 *dst1 = ring + (size_t)((ell + 1) % a.nslots) * a.slot_elems;
            const uint32_t first = tab.layer_first[ell];
            const uint32_t cnt = tab.layer_count[ell];
            for (uint32_t mi = warp; mi < cnt; mi += nwarps)
                fwd_mask_dfp<CLOW>(tab, first + mi, mi + nwarps < cnt ? first + mi + nwarps : 0xFFFFFFFFu, ell, n, src, dst1,
                             Ms, Md, lane, ci, nfl, seed0, shifts, act_x, act_y, lam, cfg_x, cfg_y, a.out, a.status,
                             a.prefetch);
            __syncthreads();
        }
    }
}

template <bool CLOW>
static auto pair_kernel_mode(int precision, int threads) {
    if (precision == COS_DF64)
        return threads <= 256 ? dp_pair_dfp_kernel<256, CLOW>
               : threads <= 384 ? dp_pair_dfp_kernel<384, CLOW>
               : threads <= 512 ? dp_pair_dfp_kernel<512, CLOW> : dp_pair_dfp_kernel<640, CLOW>;
    return threads <= 256 ? dp_pair_kernel<kMixedWidth, 256, CLOW>
           : threads <= 384 ? dp_pair_kernel<kMixedWidth, 384, CLOW>
           : threads <= 512 ? dp_pair_kernel<kMixedWidth, 512, CLOW> : dp_pair_kernel<kMixedWidth, 640, CLOW>;
}

static auto pair_kernel_for(int precision, int threads, bool clow = false) {
    return clow ? pair_kernel_mode<true>(precision, threads) : pair_kernel_mode<false>(precision, threads);
}

size_t pair_smem_bytes(int precision, int n_max) {
    const size_t msm = (size_t)n_max * n_max * kLanes;
    if (precision == COS_DF64) return 2 * msm * sizeof(df64x2);
    return ((msm * sizeof(FV<kMixedWidth>) + 15) & ~size_t(15)) + msm * sizeof(CV<kMixedWidth>);
}

size_t pair_state_bytes(int precision) { return precision == COS_DF64 ? sizeof(df64x2) : sizeof(FV<kMixedWidth>); }

int pair_width(int precision) { return precision == COS_DF64 ? 2 : kMixedWidth; }

int pair_max_active_ctas(int precision, int threads, size_t smem) {
    int nb = 0;
    auto k = pair_kernel_for(precision, threads);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, smem) == cudaSuccess ? nb : 0;
}

cos_status launch_dp_pair(Workspace *ws, const DpLaunch &L, cudaStream_t stream) {
    std::string err;
    const OrderTab *tabs = device_orders(ws->device, &err);
    if (!tabs) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    const int nfl = L.n_mat;
    const Tuning tu = get_tuning(L.n_max, L.precision, nfl);
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ws->device);
    const int nslots = 2;
    const size_t slot_elems = (size_t)host_order(L.n_max).max_slots * kLanes;
    const size_t per_cta = (size_t)nslots * slot_elems * pair_state_bytes(L.precision);
    const int cpb = pair_width(L.precision) * (kLanes / nfl);
    const int max_batches = (L.n_cfg + cpb - 1) / cpb + COS_NMAX;
    int grid = std::max(1, std::min(nsm * tu.ctas_per_sm, max_batches));
    if (ws->fixed_grid > 0) {
        grid = ws->fixed_grid;
    } else {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
            const size_t avail = ws->scratch_bytes + (size_t)(0.85 * (double)free_b);
            while (grid > 1 && (size_t)grid * per_cta > avail) grid = std::max(1, grid / 2);
        }
    }
    ws->last_grid = grid;
    cos_status st = ensure(&ws->scratch, &ws->scratch_bytes, (size_t)grid * per_cta, 1, "layer scratch");
    if (st != COS_OK) return st;
    const int threads = tu.warps * 32;
    const size_t smem = pair_smem_bytes(L.precision, L.n_max);
    auto kern = pair_kernel_for(L.precision, threads, L.clow);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "dp smem attribute");
    DpArgs a;
    memset(&a, 0, sizeof a);
    a.tabs = tabs;
    a.batches = ws->batches;
    a.n_batches = ws->plan_counts + 64;
    a.batch_list = ws->batch_list;
    a.queue = ws->queue;
    a.M = L.M;
    a.moff = L.moff;
    a.mstride = L.mstride;
    a.nf_lanes = nfl;
    a.loop_weight = (double)L.loop_weight;
    for (int l = 0; l < COS_MAX_FLAVORS; ++l) a.sigma[l] = L.sigma[l];
    a.shifts = L.shifts ? 1 : 0;
    a.absmode = L.absmode ? 1 : 0;
    a.scratch = ws->scratch;
    a.slot_elems = slot_elems;
    a.nslots = nslots;
    a.smem_n = L.n_max;
    a.prefetch = tu.prefetch;
    a.out = L.out;
    a.status = ws->status;
    e = cudaMemsetAsync(ws->queue, 0, sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e, "queue reset");
    kern<<<grid, threads, smem, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "dp launch");
    return COS_OK;
}

}  // namespace cosdp
