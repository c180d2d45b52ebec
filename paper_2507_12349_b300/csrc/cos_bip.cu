// Bipartite (two-sublattice) connected sums: the sublattice-resolved merged DP on sm_103a.
//
// Every vertex sits in a unit cell and carries a sublattice index s in {A, B} that its two
// points share; the propagator between points depends on both indices, and the connected sum
// is summed over all sublattice assignments (Methods A, strategy (i)).  Following Results A
// and Alg. 1-2, the interaction mask records the sublattice of a half-visited vertex, so the
// sum over assignments is folded into the DP:
//   mask digits  0 untouched, (1, A), (1, B), 2 full  (a full vertex forgets its sublattice)
//   state        (mu, h, s_h, v, s_v) per lane (configuration, flavor): the open loop's head
//                with its sublattice, the current endpoint with its sublattice.
// Rules (push form; the untouched-vertex factor 2 is the global 2^(n-1) as in cos_dp.cu):
//   extend  to an untouched j, for both s_j:  O(mu + (1,s_j) e_j, h, s_h, j, s_j) = sum O a(v s_v, j s_j)
//           to a half-visited j (s_j fixed):   O(mu with j full, h, s_h, j, s_j)  = sum O a(v s_v, j s_j)
//   close   C(mu) += O(mu,h,s_h,v,s_v) * sgn w a(v s_v, h s_h)
//   seed    k = min half-visited: O(mu with k full, k, s_k, k, s_k) = C(mu) in every flavor
//   sink    mu full: c = 2^(n-1) C(mu)
// Shift points ride on the shifted diagonal a(j s, j s) - sigma_{l,s} of the extension
// matrices, exactly as in the square-lattice kernel; vertex 0's shifted start seeds
// -2 sigma_{l, s_0}.
//
// Determinant weights without cycle factors (CLOW instantiations, Alg. 1 as stated for the
// SU(2) bipartite model): lanes are the two spin blocks, entering an untouched vertex has
// weight 1, the first loop (head point 0 in block 0) never steps onto vertex 0 and its close
// opens the next loop in block 1 only, every diagonal a(j s, j s) carries - alpha_{b,s} in
// both matrix copies, and the sink takes no 2^(n-1) (see cos_dp.cu for the mapping).
//
// Layout: a mask's block holds |H| x 2 rows (h, s_h) of |A| x 2 slots (v, s_v) in the
// vertex-ordered visited set; only reachable slots are written or read (a half-visited
// endpoint has its recorded sublattice, the endpoint v = h has s_h, the first loop's head has
// the recorded sublattice of vertex 0).  Lanes, persistent CTAs, the planner and the two-slot
// layer ring are those of cos_dp.cu; matrices sit in shared memory as [(v,s)][(j,t)][lane].
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "cos_dp_device.cuh"

namespace cosdp {

static __constant__ uint32_t c_p4[COS_BIP_NMAX + 2] = {1u, 4u, 16u, 64u, 256u, 1024u, 4096u, 16384u, 65536u,
                                                        262144u, 1048576u};

// ------------------------------------------------------------------ structure (host-built)

namespace {

struct BipHostOrder {
    int n = 0;
    std::vector<uint4> masks;       // {A | B << 16, S, code, off}
    std::vector<uint32_t> rank4;    // code -> block offset inside its layer
    uint32_t layer_first[kMaxLayers + 1] = {};
    uint32_t layer_count[kMaxLayers + 1] = {};
    uint32_t layer_slots[kMaxLayers + 1] = {};
    uint32_t max_slots = 0;
    uint64_t layer_work[kMaxLayers + 1] = {};   // multiply-adds of the sweep out of each layer
    cos_structure_info info{};
};

int popc_h(uint32_t x) { return __builtin_popcount(x); }

void build_bip_order(int n, BipHostOrder &o) {
    o.n = n;
    uint32_t p4[COS_BIP_NMAX + 2];
    p4[0] = 1;
    for (int i = 1; i <= n + 1; i++) p4[i] = 4 * p4[i - 1];
    const uint32_t full = (1u << n) - 1u;
    o.rank4.assign(p4[n], 0xFFFFFFFFu);
    struct Rec {
        uint4 m;
        uint64_t cost;
    };
    std::vector<std::vector<Rec>> per_layer(2 * n + 1);
    cos_structure_info &info = o.info;
    info = cos_structure_info{};
    info.n = n;
    for (uint32_t code = 0; code < p4[n]; code++) {
        uint32_t x = code, A = 0, B = 0, S = 0;
        int layer = 0;
        for (int i = 0; i < n; i++) {
            const uint32_t d = x % 4;
            x /= 4;
            if (d >= 1) A |= 1u << i;
            if (d == 3) B |= 1u << i;
            if (d == 2) S |= 1u << i;
            layer += d == 3 ? 2 : (d ? 1 : 0);
        }
        if (!(A & 1u)) continue;
        const uint32_t ones = A & ~B;
        const uint32_t H = head_set(B, ones);
        const uint32_t J = full & ~B;
        const int T = popc_h(J) + popc_h(J & ~A);
        const bool needclose = ones != 0 || B == full;
        uint64_t cost = 0;
        for (uint32_t hh = H; hh; hh &= hh - 1) {
            const int h = __builtin_ctz(hh);
            const uint32_t V = row_vmask(A, ones, h);
            const int nv = popc_h(V) + popc_h(V & B & ~(1u << h));
            const int nrows = (h == 0 && (ones & 1u)) ? 1 : 2;
            info.states += (int64_t)nrows * nv;
            info.fma_ext += (int64_t)nrows * nv * T;
            if (needclose) info.fma_close += (int64_t)nrows * nv;
            cost += (uint64_t)nrows * ((uint64_t)nv * (T + (needclose ? 1 : 0)) + 4);
            o.layer_work[layer] += (uint64_t)nrows * nv * (T + (needclose ? 1 : 0));
        }
        Rec r;
        r.m = make_uint4(A | (B << 16), S, code, 0u);
        r.cost = cost;
        per_layer[layer].push_back(r);
        info.masks++;
        info.slots += 4 * (int64_t)popc_h(H) * popc_h(A);
    }
    uint32_t first = 0;
    for (int l = 0; l <= 2 * n; l++) {
        auto &v = per_layer[l];
        std::stable_sort(v.begin(), v.end(), [](const Rec &a, const Rec &b) { return a.cost > b.cost; });
        uint32_t off = 0;
        for (auto &r : v) {
            r.m.w = off;
            o.rank4[r.m.z] = off;
            const uint32_t A = r.m.x & 0xFFFFu, B = r.m.x >> 16;
            off += 4u * (uint32_t)(popc_h(head_set(B, A & ~B)) * popc_h(A));
            o.masks.push_back(r.m);
        }
        o.layer_first[l] = first;
        o.layer_count[l] = (uint32_t)v.size();
        o.layer_slots[l] = off;
        o.max_slots = std::max(o.max_slots, off);
        first += (uint32_t)v.size();
    }
    info.max_layer_slots = o.max_slots;
}

std::mutex g_bip_mu;
BipHostOrder g_bip[COS_BIP_NMAX + 1];
bool g_bip_built[COS_BIP_NMAX + 1];

}  // namespace

struct BipOrderTab {
    const uint4 *masks;
    const uint32_t *rank4;
    uint32_t layer_first[kMaxLayers + 1];
    uint32_t layer_count[kMaxLayers + 1];
    uint32_t layer_slots[kMaxLayers + 1];
    uint32_t max_slots;
    uint32_t n;
};

namespace {

const BipHostOrder &bip_host_order(int n) {
    std::lock_guard<std::mutex> lk(g_bip_mu);
    if (!g_bip_built[n]) {
        build_bip_order(n, g_bip[n]);
        g_bip_built[n] = true;
    }
    return g_bip[n];
}

BipOrderTab *g_bip_dev[64];

const BipOrderTab *bip_device_orders(int device, std::string *err) {
    if (device < 0 || device >= 64) {
        *err = "device index out of range";
        return nullptr;
    }
    {
        std::lock_guard<std::mutex> lk(g_bip_mu);
        if (g_bip_dev[device]) return g_bip_dev[device];
    }
    BipOrderTab tabs[COS_BIP_NMAX + 1];
    memset(tabs, 0, sizeof tabs);
    for (int n = 1; n <= COS_BIP_NMAX; n++) {
        const BipHostOrder &o = bip_host_order(n);
        uint4 *dm = nullptr;
        uint32_t *dr = nullptr;
        cudaError_t e = cudaMalloc(&dm, o.masks.size() * sizeof(uint4));
        if (e == cudaSuccess) e = cudaMalloc(&dr, o.rank4.size() * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMemcpy(dm, o.masks.data(), o.masks.size() * sizeof(uint4), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dr, o.rank4.data(), o.rank4.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            *err = std::string("bipartite structure upload: ") + cudaGetErrorString(e);
            return nullptr;
        }
        BipOrderTab &t = tabs[n];
        t.masks = dm;
        t.rank4 = dr;
        memcpy(t.layer_first, o.layer_first, sizeof t.layer_first);
        memcpy(t.layer_count, o.layer_count, sizeof t.layer_count);
        memcpy(t.layer_slots, o.layer_slots, sizeof t.layer_slots);
        t.max_slots = o.max_slots;
        t.n = n;
    }
    BipOrderTab *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof tabs);
    if (e == cudaSuccess) e = cudaMemcpy(d, tabs, sizeof tabs, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        *err = std::string("bipartite structure upload: ") + cudaGetErrorString(e);
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_bip_mu);
    if (!g_bip_dev[device]) g_bip_dev[device] = d;
    return g_bip_dev[device];
}

}  // namespace

// ------------------------------------------------------------------ device code

struct BipArgs {
    const BipOrderTab *tabs;
    const int4 *batches;
    const int *n_batches;
    const int *batch_list;
    int *queue;
    const double *M;            // per configuration [n_mat][2n][2n], index (i*2 + s)*2n + (j*2 + t)
    const int64_t *moff;
    int nf_lanes;
    double loop_weight;
    double sigma2[COS_MAX_FLAVORS][2];
    int shifts;
    int absmode;
    void *scratch;              // layer ring, 8-byte elements (double or df64)
    size_t slot_elems;
    int smem_n;                 // n_max (shared-memory stride 2 n_max)
    int prefetch;
    double *out;
    int *status;
    double *csub;               // nullable (all-subsets mode): c(S) at csub[base + (S << shift)]
    const int64_t *csub_key;    // per configuration: (base << 4) | shift
};

// Extension targets of one mask, one lane per target (q < T = |J| + |J \ A|, at most 2n):
// the q-th target in (j ascending, s_j ascending) order.
//   off1 : block offset of the target mask;  meta: ai1 (bits 0-3), nA1 (4-7), s_j (8),
//   j (12-15), heads of the target mask (16-27).
// The targets are the set bits of E: bit 2j for j in J (s_j = 0, or the walk's sublattice of a
// touched j), bit 2j + 1 for an untouched j (s_j = 1), so lane q takes the (q+1)-th set bit.
__device__ __forceinline__ uint32_t spread_even(uint32_t x) {   // bit i -> bit 2i, 16 bits
    x &= 0xFFFFu;
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    return (x | (x << 1)) & 0x55555555u;
}
__device__ __forceinline__ TgtInfo bip_targets(uint32_t A, uint32_t B, uint32_t S, uint32_t J, uint32_t code,
                                               const uint32_t *__restrict__ rank4, int lane) {
    TgtInfo ti = {0u, 0u};
    const uint32_t U = J & ~A;
    if (lane < __popc(J) + __popc(U)) {
        const uint32_t E = spread_even(J) | (spread_even(U) << 1);
        const int p = (int)__fns(E, 0u, lane + 1);
        const int j = p >> 1;
        const uint32_t bj = 1u << j;
        const bool untouched = (U & bj) != 0u;
        const int sj = untouched ? (p & 1) : (int)((S >> j) & 1u);
        const uint32_t A1 = A | bj;
        const uint32_t B1 = untouched ? B : (B | bj);
        const uint32_t code1 = untouched ? code + (uint32_t)(1 + sj) * c_p4[j] : code + (uint32_t)(2 - sj) * c_p4[j];
        ti.off1 = __ldg(rank4 + code1);
        ti.meta = (uint32_t)__popc(A1 & (bj - 1u)) | ((uint32_t)__popc(A1) << 4) | ((uint32_t)sj << 8) |
                  ((uint32_t)j << 12) | (head_set(B1, A1 & ~B1) << 16);
    }
    return ti;
}

// Arithmetic of the bipartite sweep for a state type T: FP64 multiply-adds; FP32 extensions
// with the loop closes in FP64 on exactly widened states (mixed precision); or the double-float
// compensated accumulation of cos_df64.cuh (states stored as the accumulator leaves them).
//   Acc / first / mad / store: the extension dot products (state type T);
//   CT: close-matrix element, CAcc / cmad: the loop-closing sum, CV: its flavor-summed value;
//   seed: CV -> T for the next loop's first state; add: T + T (the k = 0 seed on the
//   extension's value).
template <typename T>
struct BipArith;
template <>
struct BipArith<double> {
    using Acc = double;
    using CT = double;
    using CAcc = double;
    using CV = double;
    static __device__ __forceinline__ Acc zero() { return 0.0; }
    static __device__ __forceinline__ CAcc czero() { return 0.0; }
    static __device__ __forceinline__ Acc first(double x, double y) { return x * y; }
    static __device__ __forceinline__ void mad(Acc &a, double x, double y) { a = fma(x, y, a); }
    static __device__ __forceinline__ void cmad(CAcc &a, double x, double y) { a = fma(x, y, a); }
    static __device__ __forceinline__ double store(Acc a) { return a; }
    static __device__ __forceinline__ CV close_sum(CAcc a, int nfl, int ci) { return flavor_sum(a, nfl, ci); }
    static __device__ __forceinline__ CV cadd(CV a, CV b) { return a + b; }
    static __device__ __forceinline__ double seed(CV a) { return a; }
    static __device__ __forceinline__ double add(double a, double b) { return a + b; }
    static __device__ __forceinline__ double to_double(CV a) { return a; }
};
template <>
struct BipArith<float> {
    using Acc = float;
    using CT = double;
    using CAcc = double;
    using CV = double;
    static __device__ __forceinline__ Acc zero() { return 0.0f; }
    static __device__ __forceinline__ CAcc czero() { return 0.0; }
    static __device__ __forceinline__ Acc first(float x, float y) { return x * y; }
    static __device__ __forceinline__ void mad(Acc &a, float x, float y) { a = fmaf(x, y, a); }
    static __device__ __forceinline__ void cmad(CAcc &a, float x, double y) { a = fma(widen(x), y, a); }
    static __device__ __forceinline__ float store(Acc a) { return a; }
    static __device__ __forceinline__ CV close_sum(CAcc a, int nfl, int ci) { return flavor_sum(a, nfl, ci); }
    static __device__ __forceinline__ CV cadd(CV a, CV b) { return a + b; }
    static __device__ __forceinline__ float seed(CV a) { return narrow_to(0.0f, a); }
    static __device__ __forceinline__ float add(float a, float b) { return a + b; }
    static __device__ __forceinline__ double to_double(CV a) { return a; }
};
template <>
struct BipArith<df64> {
    using Acc = DotAcc;
    using CT = df64;
    using CAcc = DotAcc;
    using CV = df64;
    static __device__ __forceinline__ Acc zero() { return DotAcc{0.0f, 0.0f}; }
    static __device__ __forceinline__ CAcc czero() { return DotAcc{0.0f, 0.0f}; }
    static __device__ __forceinline__ Acc first(df64 x, df64 y) { return dot_first(x, y); }
    static __device__ __forceinline__ void mad(Acc &a, df64 x, df64 y) { dot_add(a, x, y); }
    static __device__ __forceinline__ void cmad(CAcc &a, df64 x, df64 y) { dot_add(a, x, y); }
    static __device__ __forceinline__ df64 store(Acc a) { return df64{a.s, a.c}; }
    static __device__ __forceinline__ CV close_sum(CAcc a, int nfl, int ci) {
        return df64_flavor_sum(dot_value(a), nfl, ci);
    }
    static __device__ __forceinline__ CV cadd(CV a, CV b) { return df64_add(a, b); }
    static __device__ __forceinline__ df64 seed(CV a) { return a; }
    static __device__ __forceinline__ df64 add(df64 a, df64 b) { return df64_add(a, b); }
    static __device__ __forceinline__ double to_double(CV a) { return df64_to_double(a); }
};
// Double-float with two configurations per lane (components x, y of df64x2): the compensated
// accumulation of cos_df64.cuh in packed pairs, each component bit for bit the one-per-lane
// mode's operation.  The close runs on the extension matrices' entries (and the unshifted
// diagonal), its factor sgn w = +-2^k applied to the flavor-summed value: every step of the
// compensated sums is symmetric under negation and exact under scaling by a power of two, so
// the values are those of the one-per-lane sweep.
template <>
struct BipArith<df64x2> {
    using Acc = DotAcc2;
    using CT = df64x2;
    using CAcc = DotAcc2;
    using CV = df64x2;
    static __device__ __forceinline__ Acc zero() {
        DotAcc2 a;
        a.s = a.c = make_float2(0.0f, 0.0f);
        return a;
    }
    static __device__ __forceinline__ CAcc czero() { return zero(); }
    static __device__ __forceinline__ Acc first(const df64x2 &x, const df64x2 &y) {
        return dot_first2(x.hi, x.lo, y.hi, y.lo);
    }
    static __device__ __forceinline__ void mad(Acc &a, const df64x2 &x, const df64x2 &y) {
        dot_add2(a, x.hi, x.lo, y.hi, y.lo);
    }
    static __device__ __forceinline__ void cmad(CAcc &a, const df64x2 &x, const df64x2 &y) {
        dot_add2(a, x.hi, x.lo, y.hi, y.lo);
    }
    static __device__ __forceinline__ df64x2 store(const Acc &a) {
        df64x2 r;
        r.hi = a.s;
        r.lo = a.c;
        return r;
    }
    static __device__ __forceinline__ CV close_sum(const CAcc &a, int nfl, int ci) {
        return dfpair(df64_flavor_sum(dot_value(DotAcc{a.s.x, a.c.x}), nfl, ci),
                      df64_flavor_sum(dot_value(DotAcc{a.s.y, a.c.y}), nfl, ci));
    }
    static __device__ __forceinline__ CV cadd(const CV &a, const CV &b) {
        return dfpair(df64_add(dfx(a), dfx(b)), df64_add(dfy(a), dfy(b)));
    }
    static __device__ __forceinline__ df64x2 seed(const CV &a) { return a; }
    static __device__ __forceinline__ df64x2 add(const df64x2 &a, const df64x2 &b) { return cadd(a, b); }
};

// Mixed mode with two configurations per lane (components x, y): the extensions as packed FP32
// pairs (each component bit for bit the one-per-lane mode's operation); the closes as the
// square-lattice mixed sweep takes them, compensated FP32 sums (close_add2: Dot2 on close
// matrices split into FP32 pairs hi + lo) widened and added in FP64 once per mask, so the FP64
// pipe carries no per-state work.  No to_double: the sweep writes each component's output.
template <>
struct BipArith<float2> {
    using Acc = float2;
    using CT = df64x2;     // close matrices sgn w M split into FP32 pairs, per configuration
    using CAcc = DotAcc2;
    using CV = double2;
    static __device__ __forceinline__ Acc zero() { return make_float2(0.0f, 0.0f); }
    static __device__ __forceinline__ CAcc czero() {
        DotAcc2 a;
        a.s = a.c = make_float2(0.0f, 0.0f);
        return a;
    }
    static __device__ __forceinline__ Acc first(float2 x, float2 y) { return mul2(x, y); }
    static __device__ __forceinline__ void mad(Acc &a, float2 x, float2 y) { a = fma2(x, y, a); }
    static __device__ __forceinline__ void cmad(CAcc &a, float2 x, const df64x2 &y) { close_add2(a, x, y.hi, y.lo); }
    static __device__ __forceinline__ float2 store(Acc a) { return a; }
    static __device__ __forceinline__ CV close_sum(const CAcc &a, int nfl, int ci) {
        return make_double2(flavor_sum(close_value(DotAcc{a.s.x, a.c.x}), nfl, ci),
                            flavor_sum(close_value(DotAcc{a.s.y, a.c.y}), nfl, ci));
    }
    static __device__ __forceinline__ CV cadd(CV a, CV b) { return make_double2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ float2 seed(CV a) {
        return make_float2(narrow_to(0.0f, a.x), narrow_to(0.0f, a.y));
    }
    static __device__ __forceinline__ float2 add(float2 a, float2 b) { return add2(a, b); }
};

// Loads of a matrix entry at a shared-memory byte address (the rows keep one 32-bit address
// per state, so an entry costs one add).
template <typename T>
__device__ __forceinline__ T lds_as(uint32_t a);
template <>
__device__ __forceinline__ float lds_as<float>(uint32_t a) {
    float r;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(r) : "r"(a));
    return r;
}
template <>
__device__ __forceinline__ double lds_as<double>(uint32_t a) {
    double r;
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(r) : "r"(a));
    return r;
}
template <>
__device__ __forceinline__ df64 lds_as<df64>(uint32_t a) {
    df64 r;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(r.hi), "=f"(r.lo) : "r"(a));
    return r;
}

template <>
__device__ __forceinline__ float2 lds_as<float2>(uint32_t a) {
    float2 r;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "r"(a));
    return r;
}

template <>
__device__ __forceinline__ df64x2 lds_as<df64x2>(uint32_t a) {
    df64x2 r;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r.hi.x), "=f"(r.hi.y), "=f"(r.lo.x), "=f"(r.lo.y)
                 : "r"(a));
    return r;
}

template <typename T, bool BYTE>
__device__ __forceinline__ T ms_at(const T *Ms, uint32_t a) {
    if constexpr (BYTE) return lds_as<T>(a);
    else return Ms[a];
}

// One row (mu, h, s_h): NV reachable endpoint states, the close, every extension.
template <typename T, int NV>
__device__ __forceinline__ void bip_row(const T *__restrict__ src, T *__restrict__ dst1, const T *__restrict__ Ms,
                                        const typename BipArith<T>::CT *__restrict__ Md, const TgtInfo &ti, int nT,
                                        uint32_t Vrow, uint32_t A, uint32_t B, uint32_t S, uint32_t rowbase, int h,
                                        int sh, int n2, bool needclose, int lane, typename BipArith<T>::CAcc &csum) {
    using Ar = BipArith<T>;
    // The row's endpoint states (v, s_v) in ascending order are the set bits 2 v + s_v of R: a
    // half-visited v on its own sublattice, v = h on s_h, any other (full) v on both.
    const uint32_t ones = A & ~B;
    const uint32_t bh = 1u << h;
    const uint32_t vhalf = Vrow & ones;
    uint32_t R = spread_even(Vrow & ~ones & ~bh) * 3u | spread_even(vhalf & ~S) | (spread_even(vhalf & S) << 1);
    if (Vrow & ~ones & bh) R |= 1u << (2 * h + sh);
    using CT = typename Ar::CT;
    // Matrix entries by shared-memory byte address (mixed, double-float: one add per entry) or,
    // in FP64 where that measured no better, by element index: ra[t] locates Ms[(v_t, s_t)][0]
    // of this lane in units of kU bytes from kBase.
    constexpr bool kByte = !std::is_same<T, double>::value;
    constexpr uint32_t kU = kByte ? (uint32_t)sizeof(T) : 1u;
    const uint32_t msb = kByte ? (uint32_t)__cvta_generic_to_shared(Ms) : 0u;
    T o[NV];
    uint32_t ra[NV];
    if constexpr (std::is_same<T, float>::value) {
        // mixed, one configuration per lane: lane t decodes state t once per row, the loop
        // shuffles it (such rows are short in issue time, so the per-state chain below would
        // lead them)
        uint32_t lslot = 0u;
        int lrs = 0;
        if (lane < NV) {
            const int p = (int)__fns(R, 0u, lane + 1);   // 2 v + s_v of state `lane`
            lslot = rowbase + (uint32_t)(__popc(A & ((1u << (p >> 1)) - 1u)) * 2 + (p & 1));
            lrs = p * n2 * kLanes;
        }
        const uint32_t mlane = msb + (uint32_t)lane * kU;
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            const uint32_t sl = __shfl_sync(0xFFFFFFFFu, lslot, t);
            ra[t] = mlane + (uint32_t)__shfl_sync(0xFFFFFFFFu, lrs, t) * kU;
            o[t] = src[(size_t)sl * kLanes + lane];
        }
    } else {
        // FP64, double-float and mixed with two configurations per lane: the set bits of R in
        // turn (a short branch-free chain per state)
        uint32_t rr = R;
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            const int p = __ffs(rr) - 1;
            rr &= rr - 1u;
            const uint32_t sl = rowbase + (uint32_t)(__popc(A & ((1u << (p >> 1)) - 1u)) * 2 + (p & 1));
            ra[t] = msb + (uint32_t)(p * n2 * kLanes + lane) * kU;
            o[t] = src[(size_t)sl * kLanes + lane];
        }
    }
    if (needclose) {
        const uint32_t hc = (uint32_t)((h * 2 + sh) * kLanes);
        if constexpr (std::is_same<T, df64x2>::value) {
            // the close on the extension matrices' column (h, s_h), except the head's own state,
            // whose entry is the unshifted diagonal kept apart in Md[(h, s_h)][lane]; the sign
            // sgn w comes after the flavor sum
            const uint32_t own = msb + (uint32_t)((h * 2 + sh) * n2 * kLanes + lane) * kU;
            const uint32_t dga = (uint32_t)__cvta_generic_to_shared(Md) + (hc + (uint32_t)lane) * kU;
#pragma unroll
            for (int t = 0; t < NV; ++t)
                Ar::cmad(csum, o[t], lds_as<CT>(ra[t] == own ? dga : ra[t] + hc * kU));
        } else if constexpr (kByte) {
            // Md[(v,s)][(h,s_h)] at md + (ra - msb) kr + (h 2 + s_h) 32 sizeof(CT), kr = sizeof(CT) / sizeof(T)
            constexpr uint32_t kr = sizeof(CT) / sizeof(T);
            const uint32_t dmd = (uint32_t)__cvta_generic_to_shared(Md) - kr * msb + hc * (uint32_t)sizeof(CT);
#pragma unroll
            for (int t = 0; t < NV; ++t) Ar::cmad(csum, o[t], lds_as<CT>(kr * ra[t] + dmd));
        } else {
#pragma unroll
            for (int t = 0; t < NV; ++t) Ar::cmad(csum, o[t], Md[ra[t] + hc]);
        }
    }
    // this row's target slots, lane-parallel: off1 + ((hidx1 * 2 + s_h) * nA1 + ai1) * 2 + s_j
    const uint32_t hlow = (1u << h) - 1u;
    const uint32_t ai1 = ti.meta & 15u, nA1 = (ti.meta >> 4) & 15u, sj1 = (ti.meta >> 8) & 1u;
    const uint32_t hi1 = (uint32_t)__popc((ti.meta >> 16) & hlow);
    const uint32_t tslot = ti.off1 + ((hi1 * 2u + (uint32_t)sh) * nA1 + ai1) * 2u + sj1;
    // and their matrix columns (j, s_j) in the units of ra: formed lane-parallel here for the
    // byte-addressed rows, decoded per target from the shuffled meta in FP64 (measured better
    // there)
    const uint32_t tcol = (((ti.meta >> 12) & 15u) * 2u + sj1) * (kLanes * kU);
    auto column = [&](int qq) -> uint32_t {
        if constexpr (kByte) return __shfl_sync(0xFFFFFFFFu, tcol, qq);
        const uint32_t m = __shfl_sync(0xFFFFFFFFu, ti.meta, qq);
        return (((m >> 12) & 15u) * 2u + ((m >> 8) & 1u)) * (kLanes * kU);
    };
    int q = 0;
    for (; q + 1 < nT; q += 2) {
        const uint32_t ca = column(q);
        const uint32_t cb = column(q + 1);
        typename Ar::Acc da = Ar::first(o[0], ms_at<T, kByte>(Ms, ra[0] + ca));
        typename Ar::Acc db = Ar::first(o[0], ms_at<T, kByte>(Ms, ra[0] + cb));
#pragma unroll
        for (int t = 1; t < NV; ++t) {
            Ar::mad(da, o[t], ms_at<T, kByte>(Ms, ra[t] + ca));
            Ar::mad(db, o[t], ms_at<T, kByte>(Ms, ra[t] + cb));
        }
        const uint32_t sa = __shfl_sync(0xFFFFFFFFu, tslot, q);
        const uint32_t sb = __shfl_sync(0xFFFFFFFFu, tslot, q + 1);
        dst1[(size_t)sa * kLanes + lane] = Ar::store(da);
        dst1[(size_t)sb * kLanes + lane] = Ar::store(db);
    }
    if (q < nT) {
        const uint32_t ca = column(q);
        typename Ar::Acc da = Ar::first(o[0], ms_at<T, kByte>(Ms, ra[0] + ca));
#pragma unroll
        for (int t = 1; t < NV; ++t) Ar::mad(da, o[t], ms_at<T, kByte>(Ms, ra[t] + ca));
        const uint32_t sa = __shfl_sync(0xFFFFFFFFu, tslot, q);
        dst1[(size_t)sa * kLanes + lane] = Ar::store(da);
    }
}

template <typename T>
__device__ __forceinline__ void bip_row_dispatch(int nv, const T *src, T *dst1, const T *Ms,
                                                 const typename BipArith<T>::CT *Md, const TgtInfo &ti, int nT,
                                                 uint32_t Vrow, uint32_t A, uint32_t B, uint32_t S, uint32_t rowbase,
                                                 int h, int sh, int n2, bool needclose, int lane,
                                                 typename BipArith<T>::CAcc &csum) {
#define COS_BROW(K)                                                                                            \
    case K:                                                                                                    \
        bip_row<T, K>(src, dst1, Ms, Md, ti, nT, Vrow, A, B, S, rowbase, h, sh, n2, needclose, lane, csum);    \
        break;
    switch (nv) {
        COS_BROW(1)
        COS_BROW(2)
        COS_BROW(3)
        COS_BROW(4)
        COS_BROW(5)
        COS_BROW(6)
        COS_BROW(7)
        COS_BROW(8)
        COS_BROW(9)
        COS_BROW(10)
        COS_BROW(11)
        COS_BROW(12)
        COS_BROW(13)
        COS_BROW(14)
        COS_BROW(15)
        COS_BROW(16)
        COS_BROW(17)
        default:
            break;
    }
#undef COS_BROW
}

// One interaction mask: its rows, the flavor sum of the close, the seed of the next loop or
// the sink.  seedsh = sgn 2 sigma_{l, s} of this lane for vertex 0's shifted start on s.
// SUB: all-subsets mode.  A mask with no half-visited vertex closes the connected covers of
// its full set B (times 2^(|B|-1) for cycle factors); its close is stored at csub[B << cshift]
// (csub: this lane's output base, valid on active lanes), also where the sweep itself drops it.
template <typename T, bool CLOW, bool SUB = false>
__device__ __forceinline__ void bip_mask(const BipOrderTab &tab, uint32_t mask_index, uint32_t next_index, int ell,
                                         int n, const T *src, T *dst1, const T *Ms,
                                         const typename BipArith<T>::CT *Md, int lane, int ci, int nfl,
                                         const typename BipArith<T>::CV seedsh[2], bool shifts, bool active, int lam,
                                         int cfg, double *out, int *status, int prefetch, double *csub = nullptr,
                                         int cshift = 0, int cfg1 = -1, float cfac2 = 1.0f) {
    using Ar = BipArith<T>;
    const uint32_t full = (1u << n) - 1u;
    const uint4 mk = __ldg(tab.masks + mask_index);
    const uint32_t A = mk.x & 0xFFFFu, B = mk.x >> 16, S = mk.y, code = mk.z, off = mk.w;
    const uint32_t ones = A & ~B;
    const uint32_t H = head_set(B, ones);
    const uint32_t J = full & ~B & (CLOW ? ~(ones & 1u) : 0xFFFFFFFFu);   // CLOW: not onto the head point
    const int nA = __popc(A);
    const bool dead = (ones == 0u) && (B != full);
    const bool needclose = !dead || SUB;
    if (prefetch > 0 && next_index != 0xFFFFFFFFu) {
        const uint4 nk = __ldg(tab.masks + next_index);
        const uint32_t nA_ = nk.x & 0xFFFFu, nB_ = nk.x >> 16;
        prefetch_block(src, nk.w,
                       4u * (uint32_t)(__popc(head_set(nB_, nA_ & ~nB_)) * __popc(nA_)), lane, prefetch);
    }
    const TgtInfo ti = bip_targets(A, B, S, J, code, tab.rank4, lane);
    const int nT = __popc(J) + __popc(J & ~A);
    const int n2 = 2 * n;
    typename Ar::CAcc csum = Ar::czero();
    for (uint32_t hh = H; hh; hh &= hh - 1u) {
        const int h = __ffs(hh) - 1;
        const int hidx = __popc(H & ((1u << h) - 1u));
        const uint32_t Vrow = row_vmask(A, ones, h);
        const int nv = __popc(Vrow) + __popc(Vrow & B & ~(1u << h));
        const bool first_loop = (h == 0) && (ones & 1u);
        const int sh0 = first_loop ? (int)(S & 1u) : 0;
        const int sh1 = first_loop ? sh0 : 1;
        for (int sh = sh0; sh <= sh1; ++sh) {
            const uint32_t rowbase = off + (uint32_t)((hidx * 2 + sh) * nA * 2);
            bip_row_dispatch<T>(nv, src, dst1, Ms, Md, ti, nT, Vrow, A, B, S, rowbase, h, sh, n2, needclose, lane,
                                csum);
        }
    }
    if (!needclose) return;   // no half-visited vertex and not full: disconnected, dropped
    typename Ar::CV C = Ar::close_sum(csum, nfl, ci);
    if constexpr (std::is_same<T, df64x2>::value) {   // the close's factor sgn w = cfac2 (see BipArith<df64x2>)
        if (cfac2 != 1.0f) {
            const float2 f = make_float2(cfac2, cfac2);
            C.hi = mul2(C.hi, f);
            C.lo = mul2(C.lo, f);
        }
    }
    if constexpr (SUB) {
        if (ones == 0u) {
            if (active && lam == 0) {
                const double c = Ar::to_double(C);
                csub[(int64_t)B << cshift] = CLOW ? c : ldexp(c, __popc(B) - 1);
            }
            if (dead) return;
        }
    }
    if (ones) {
        const int k = __ffs(ones) - 1;
        const uint32_t bk = 1u << k;
        const int sk = (int)((S >> k) & 1u);
        const uint32_t B1 = B | bk;
        const uint32_t code1 = code + (uint32_t)(2 - sk) * c_p4[k];
        const int hi1 = __popc(head_set(B1, A & ~B1) & (bk - 1u));
        const uint32_t off1 = __ldg(tab.rank4 + code1);
        T *tp = dst1 + (size_t)(off1 + (uint32_t)(((hi1 * 2 + sk) * nA + __popc(A & (bk - 1u))) * 2 + sk)) * kLanes +
                lane;
        typename Ar::CV val = C;
        if (!CLOW && ell == 1 && shifts) val = Ar::cadd(val, seedsh[S & 1u]);   // vertex 0 carries a shift point
        const T tv = Ar::seed(val);                                              // (mixed: rounded to FP32)
        if (CLOW) *tp = (k == 0 && lam == 0) ? Ar::store(Ar::zero()) : tv;      // k = 0: block 1 only
        else if (k == 0) *tp = Ar::add(*tp, tv);                                 // the extension into 0' wrote it
        else *tp = tv;
    } else if (active && (lam == 0) && out) {
        if constexpr (std::is_same<T, float2>::value || std::is_same<T, df64x2>::value) {
            // cfg1: the lane's second configuration, or -1
            double v0, v1;
            if constexpr (std::is_same<T, float2>::value) {
                v0 = C.x;
                v1 = C.y;
            } else {
                v0 = df64_to_double(dfx(C));
                v1 = df64_to_double(dfy(C));
            }
            const double c0 = CLOW ? v0 : ldexp(v0, n - 1);
            out[cfg] = c0;
            bool fin = isfinite(c0);
            if (cfg1 >= 0) {
                const double c1 = CLOW ? v1 : ldexp(v1, n - 1);
                out[cfg1] = c1;
                fin = fin && isfinite(c1);
            }
            if (!fin) atomicOr(status, kStatusNonFinite);
        } else {
            const double c = CLOW ? Ar::to_double(C) : ldexp(Ar::to_double(C), n - 1);
            out[cfg] = c;
            if (!isfinite(c)) atomicOr(status, kStatusNonFinite);
        }
    }
}

// An element of the matrices or states from the values of the lane's configurations: the
// packed mixed types take both (x, y), the one-per-lane types the first.
template <typename T>
__device__ __forceinline__ void to_elem2(double x0, double, T &r) {
    to_elem(x0, r);
}
__device__ __forceinline__ void to_elem2(double x0, double x1, float2 &r) {
    r = make_float2((float)x0, (float)x1);
}
__device__ __forceinline__ void to_elem2(double x0, double x1, double2 &r) { r = make_double2(x0, x1); }
__device__ __forceinline__ void to_elem2(double x0, double x1, df64x2 &r) { r = dfpair(df64_from(x0), df64_from(x1)); }

template <typename T, bool CLOW, bool SUB = false>
__global__ void __launch_bounds__(512, 1) dp_bip_kernel(const __grid_constant__ BipArgs a) {
    extern __shared__ __align__(16) unsigned char smem_bip[];
    __shared__ int s_batch;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int nsm = 4 * a.smem_n * a.smem_n * kLanes;
    using CT = typename BipArith<T>::CT;
    T *Ms = reinterpret_cast<T *>(smem_bip);   // extension matrices, shifted diagonal
    CT *Md = reinterpret_cast<CT *>(smem_bip + ((nsm * sizeof(T) + 15) & ~size_t(15)));   // close: sgn w M
    T *ring = reinterpret_cast<T *>(a.scratch) + (size_t)blockIdx.x * 2 * a.slot_elems;
    const int nfl = a.nf_lanes;
    const int lam = lane % nfl;
    const int ci = lane / nfl;
    const double sgn = a.absmode ? 1.0 : -1.0;
    double sig[2];
    typename BipArith<T>::CV seedsh[2];
    for (int s = 0; s < 2; ++s) {
        sig[s] = a.absmode ? fabs(a.sigma2[lam][s]) : a.sigma2[lam][s];
        to_elem2(sgn * 2.0 * sig[s], sgn * 2.0 * sig[s], seedsh[s]);
    }
    const bool shifts = a.shifts != 0;
    const int nbatch = *a.n_batches;
    // two configurations per lane (mixed float2, double-float df64x2): the second sits cpl
    // places after the first.  Double-float keeps only the close's diagonal in Md and applies
    // the close's factor sgn w = +-2^k (loop weight a power of two) per mask.
    constexpr bool kPair = std::is_same<T, float2>::value || std::is_same<T, df64x2>::value;
    constexpr bool kDiagClose = std::is_same<T, df64x2>::value;
    const int cpl = kLanes / nfl;
    const float cfac2 = (float)(sgn * a.loop_weight);   // +-2^k: applied exactly (double-float, two per lane)
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_batch = atomicAdd(a.queue, 1);
        __syncthreads();
        const int b = s_batch;
        if (b >= nbatch) break;
        const int4 bd = a.batches[b];
        const int n = bd.x;
        const BipOrderTab &tab = a.tabs[n];
        const bool active = (ci < bd.z) && (ci * nfl + nfl <= kLanes);
        const int cfg = active ? a.batch_list[bd.y + ci] : -1;
        const bool active1 = kPair && active && (ci + cpl < bd.z);
        const int cfg1 = active1 ? a.batch_list[bd.y + cpl + ci] : -1;
        const int n2 = 2 * n;
        const double *Mc = nullptr, *Mc1 = nullptr;
        if (active) Mc = a.M + a.moff[cfg] + (size_t)lam * n2 * n2;
        if (active1) Mc1 = a.M + a.moff[cfg1] + (size_t)lam * n2 * n2;
        double *cs = nullptr;
        int csh = 0;
        if (SUB && active) {
            const int64_t key = a.csub_key[cfg];
            cs = a.csub + (key >> 4);
            csh = (int)(key & 15);
        }
        const double cfac = sgn * a.loop_weight;
        for (int e = warp; e < n2 * n2; e += nwarps) {
            double val = active ? Mc[e] : 0.0;
            double val1 = active1 ? Mc1[e] : 0.0;
            if (a.absmode) {
                val = fabs(val);
                val1 = fabs(val1);
            }
            const int r = e / n2, c = e % n2;
            if (CLOW) {
                const double d = (r == c) ? sgn * sig[r & 1] : 0.0;   // a(j s, j s) - alpha_{b,s}
                const double m = (r == c) ? val + d : val, m1 = (r == c) ? val1 + d : val1;
                to_elem2(m, m1, Ms[e * kLanes + lane]);
                if constexpr (kDiagClose) {
                    if (r == c) to_elem2(m, m1, Md[r * kLanes + lane]);
                } else {
                    to_elem2(cfac * m, cfac * m1, Md[e * kLanes + lane]);
                }
            } else {
                const bool shifted = (r == c) && (r >= 2) && shifts;   // (j, s) -> (j, s), j >= 1
                const double d = sgn * sig[r & 1];
                to_elem2(shifted ? val + d : val, shifted ? val1 + d : val1, Ms[e * kLanes + lane]);
                if constexpr (kDiagClose) {
                    if (r == c) to_elem2(val, val1, Md[r * kLanes + lane]);   // unshifted
                } else {
                    to_elem2(cfac * val, cfac * val1, Md[e * kLanes + lane]);
                }
            }
        }
        // Start: the loop through the normal point of vertex 0 on sublattice s_0 (layer 1,
        // masks mu_0 = (1, A) and (1, B); row (0, s_0), endpoint (0, s_0)).
        if (warp == 0) {
            for (int s0 = 0; s0 < 2; ++s0) {
                const uint32_t off = __ldg(tab.rank4 + 1 + s0);
                const double one = (CLOW && lam != 0) ? 0.0 : 1.0;
                to_elem2(one, one, ring[(size_t)(1 & 1) * a.slot_elems + (size_t)(off + 3u * (uint32_t)s0) * kLanes + lane]);
            }
        }
        __syncthreads();
        for (int ell = 1; ell <= 2 * n; ++ell) {
            const T *src = ring + (size_t)(ell & 1) * a.slot_elems;
            T *dst1 = ring + (size_t)((ell + 1) & 1) * a.slot_elems;
            const uint32_t first = tab.layer_first[ell];
            const uint32_t cnt = tab.layer_count[ell];
            for (uint32_t mi = warp; mi < cnt; mi += nwarps)
                bip_mask<T, CLOW, SUB>(tab, first + mi, mi + nwarps < cnt ? first + mi + nwarps : 0xFFFFFFFFu, ell, n, src,
                                       dst1, Ms, Md, lane, ci, nfl, seedsh, shifts, active, lam, cfg, a.out, a.status,
                                       a.prefetch, cs, csh, cfg1, cfac2);
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------ launch

struct BipLaunch {
    int n_cfg = 0;
    int n_max = 0;
    const int32_t *order = nullptr;
    const double *M = nullptr;
    const int64_t *moff = nullptr;
    int n_mat = 1;
    int loop_weight = 1;
    double sigma2[COS_MAX_FLAVORS][2] = {};
    bool shifts = false;
    double *out = nullptr;
    bool absmode = false;
    int precision = COS_FP64;
    bool clow = false;   // determinant weights without cycle factors (n_mat = 2 spin blocks)
    double *csub = nullptr;              // all-subsets mode (FP64): see BipArgs
    const int64_t *csub_key = nullptr;
    bool allow_empty = false;            // order 0 = empty derived problem (skipped by the planner)
};

// Largest n_max of the two-configurations-per-lane sweeps: their matrices (4 n^2 entries per
// lane) fill 192 KB of shared memory at n = 8 (mixed: FP32 pairs, close matrices split into
// FP32 hi + lo pairs) or 136 KB (double-float: df64 pairs, the closes on them and a diagonal
// of 2n pairs).
constexpr int kBipPairMaxN = 8;

// Configurations per lane of a launch: two for the mixed sweep and, at a loop weight that is a
// power of two (the close's factor sgn w applied exactly), the double-float sweep up to
// kBipPairMaxN; else one.
static int bip_lane_width(const BipLaunch &L) {
    if (L.csub || L.n_max > kBipPairMaxN) return 1;
    if (L.precision == COS_MIXED) return 2;
    const bool pow2 = L.loop_weight >= 1 && (L.loop_weight & (L.loop_weight - 1)) == 0;
    return (L.precision == COS_DF64 && pow2) ? 2 : 1;
}

static cos_status launch_bip(Workspace *ws, const BipLaunch &L, cudaStream_t stream) {
    std::string err;
    const BipOrderTab *tabs = bip_device_orders(ws->device, &err);
    if (!tabs) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ws->device);
    const size_t slot_elems = (size_t)bip_host_order(L.n_max).max_slots * kLanes;
    const int width = bip_lane_width(L);
    const bool dfpair_sweep = width == 2 && L.precision == COS_DF64;
    const size_t per_cta = 2 * slot_elems * (dfpair_sweep ? 16 : sizeof(double));   // state bytes per lane
    const int cpb = width * (kLanes / L.n_mat);
    const int max_batches = (L.n_cfg + cpb - 1) / cpb + COS_NMAX;
    int grid = std::max(1, std::min(nsm, max_batches));
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
        const size_t avail = ws->scratch_bytes + (size_t)(0.85 * (double)free_b);
        while (grid > 1 && (size_t)grid * per_cta > avail) grid = std::max(1, grid / 2);
    }
    ws->last_grid = grid;
    cos_status st = ensure(&ws->scratch, &ws->scratch_bytes, (size_t)grid * per_cta, 1, "bipartite layer scratch");
    if (st != COS_OK) return st;
    // extension matrices in the state type, close matrices in FP64 (double-float for df64), per
    // configuration of the lane
    const size_t mel = (size_t)4 * L.n_max * L.n_max * kLanes;
    const size_t es = width * (L.precision == COS_MIXED ? sizeof(float) : sizeof(double));
    const size_t close_bytes =
        dfpair_sweep ? (size_t)2 * L.n_max * kLanes * sizeof(df64x2) : mel * width * sizeof(double);
    const size_t smem = ((mel * es + 15) & ~size_t(15)) + close_bytes;
    auto kern = L.csub                     ? (L.clow ? dp_bip_kernel<double, true, true> : dp_bip_kernel<double, false, true>)
                : dfpair_sweep             ? (L.clow ? dp_bip_kernel<df64x2, true> : dp_bip_kernel<df64x2, false>)
                : width == 2               ? (L.clow ? dp_bip_kernel<float2, true> : dp_bip_kernel<float2, false>)
                : L.precision == COS_DF64  ? (L.clow ? dp_bip_kernel<df64, true> : dp_bip_kernel<df64, false>)
                : L.precision == COS_MIXED ? (L.clow ? dp_bip_kernel<float, true> : dp_bip_kernel<float, false>)
                                           : (L.clow ? dp_bip_kernel<double, true> : dp_bip_kernel<double, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "bipartite smem attribute");
    BipArgs a;
    memset(&a, 0, sizeof a);
    a.tabs = tabs;
    a.batches = ws->batches;
    a.n_batches = ws->plan_counts + 64;
    a.batch_list = ws->batch_list;
    a.queue = ws->queue;
    a.M = L.M;
    a.moff = L.moff;
    a.nf_lanes = L.n_mat;
    a.loop_weight = (double)L.loop_weight;
    memcpy(a.sigma2, L.sigma2, sizeof a.sigma2);
    a.shifts = L.shifts ? 1 : 0;
    a.absmode = L.absmode ? 1 : 0;
    a.scratch = ws->scratch;
    a.slot_elems = slot_elems;
    a.smem_n = L.n_max;
    // an L2 prefetch of the next mask's rows pays only with 4-byte states (mixed, one per lane:
    // +1.6 %); with 8-byte states it costs (double-float -3.7 %, FP64 -0.4 %, mixed two per lane
    // -1 %, order 8)
    a.prefetch = (L.precision == COS_MIXED && width == 1) ? 1 : 0;
    a.out = L.out;
    a.status = ws->status;
    a.csub = L.csub;
    a.csub_key = L.csub_key;
    e = cudaMemsetAsync(ws->queue, 0, sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e, "queue reset");
    kern<<<grid, 512, smem, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "bipartite dp launch");
    return COS_OK;
}

static cos_status run_bip(Workspace *ws, BipLaunch L, double *d_abs_mass, cudaStream_t stream) {
    cos_status st = launch_plan_batches(ws, L.n_cfg, L.n_max, L.order, bip_lane_width(L) * (kLanes / L.n_mat), stream,
                                        L.allow_empty);
    if (st != COS_OK) return st;
    st = launch_bip(ws, L, stream);
    if (st != COS_OK || !d_abs_mass) return st;
    L.out = d_abs_mass;
    L.absmode = true;
    return launch_bip(ws, L, stream);
}

static cos_status check_bip(int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff, int n_mat,
                            int loop_weight, const double *d_M4, cos_precision precision, const double *d_out,
                            const char *fn) {
    if (n_cfg < 0 || n_mat < 1 || n_mat > COS_MAX_FLAVORS || loop_weight < 1) {
        set_error(std::string(fn) + ": n_cfg < 0, n_mat outside [1, 8] or loop_weight < 1");
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
    if (n_cfg > 0 && (!d_order || !d_moff || !d_M4 || !d_out)) {
        set_error(std::string(fn) + ": null device pointer");
        return COS_ERR_ARG;
    }
    return COS_OK;
}

cos_status bip_matrices_body(Workspace *ws, int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                             int n_mat, int loop_weight, const double *h_sigma2, const double *d_M4,
                             cos_precision precision, double *d_out, double *d_abs_mass, cudaStream_t stream,
                             bool clow) {
    BipLaunch L;
    L.clow = clow;
    L.precision = precision;
    L.n_cfg = n_cfg;
    L.n_max = n_max;
    L.order = d_order;
    L.M = d_M4;
    L.moff = d_moff;
    L.n_mat = n_mat;
    L.loop_weight = loop_weight;
    for (int l = 0; l < n_mat; ++l)
        for (int s = 0; s < 2; ++s) {
            L.sigma2[l][s] = h_sigma2 ? h_sigma2[l * 2 + s] : 0.0;
            if (L.sigma2[l][s] != 0.0) L.shifts = true;
        }
    L.out = d_out;
    return run_bip(ws, L, d_abs_mass, stream);
}

cos_status bip_subsets_dp(Workspace *ws, int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                          int n_mat, int loop_weight, const double *h_sigma2, const double *d_M4, bool clow,
                          double *d_csub, const int64_t *d_csub_key, bool allow_empty, cudaStream_t stream) {
    BipLaunch L;
    L.clow = clow;
    L.precision = COS_FP64;
    L.n_cfg = n_cfg;
    L.n_max = n_max;
    L.order = d_order;
    L.M = d_M4;
    L.moff = d_moff;
    L.n_mat = n_mat;
    L.loop_weight = loop_weight;
    for (int l = 0; l < n_mat; ++l)
        for (int s = 0; s < 2; ++s) {
            L.sigma2[l][s] = h_sigma2 ? h_sigma2[l * 2 + s] : 0.0;
            if (L.sigma2[l][s] != 0.0) L.shifts = true;
        }
    L.csub = d_csub;
    L.csub_key = d_csub_key;
    L.allow_empty = allow_empty;
    return run_bip(ws, L, nullptr, stream);
}

// ------------------------------------------------------------------ reverse (adjoint) sweep
// Gradient of the bipartite sums, the adjoint of the sweep above (as cos_adjoint.cu is of the
// square one).  Per batch the CTA re-runs the forward sweep keeping every layer at its place
// (checkpointed where memory binds, the segments re-run before they are reversed), then walks
// the layers backwards with Obar = dc/dO, each adjoint overwriting its forward state:
//   Obar(mu,h,s_h,v,s_v) = sum_q D_q Ms[(v,s_v)][(j_q,s_q)] + Cbar Md[(v,s_v)][(h,s_h)],
//   dM[(v,s_v)][(j_q,s_q)] += D_q O,  dM[(v,s_v)][(h,s_h)] += sgn w Cbar O,
// D_q = Obar of extension target q (the forward's target table), Cbar = the flavor sum of the
// seed slot's Obar (or gout 2^(n-1) at the full mask).  Shift weights: the shifted diagonal
// (v,s) -> (v,s) for half-visited v >= 1 gives dsigma_{l,s} = sgn sum_v (the extension part of
// dM[(v,s)][(v,s)], the closes' diagonal terms kept apart), read once per batch, plus the
// shifted start sgn 2 Obar(seed) read from layer 2 at the end of the batch.  Determinant weights (CLOW): the Alg. 1 sweep, the k = 0 close
// seeded block 1 only, Cbar(full) = gout, and dalpha_{b,s} = -sum_j dM_b[(j,s)][(j,s)].
// Warps own endpoint units (v, s_v), unit v * 2 + s_v modulo the warp count (2n warps, at most
// 16): one writer per dM row, no atomics.  Shared memory holds Ms, Md and dM, 3 x 4 n^2 doubles
// per lane, so one CTA per SM; at order 9 dM moves to the CTA's global scratch.
// Storage as in the square adjoint (cos_adjoint.cu): each adjoint overwrites the forward state
// it is formed from, and where memory binds the layers are checkpointed and the segments between
// two checkpoints re-run from the first before they are reversed.
struct BipAdjArgs {
    BipArgs f;
    size_t store_elems;     // layer storage per CTA (checkpoint + segment areas) * 32
    size_t cta_elems;       // store_elems, plus the dM accumulators when they live in global memory
    uint32_t ckmask[COS_BIP_NMAX + 1];   // per order: bit l = layer l is a checkpoint
    const double *gout;
    double *gM;             // NULL or dLoss/dM4, layout of M4
    double *gsig;           // NULL or [n_cfg][n_mat][2]
    int dm_global;          // dM in the CTA's global scratch (after the adjoint slots), not shared memory
};

// Targets q in [Q0, Q1) of one endpoint (v, s_v): loads first, then the multiply-adds.
template <int Q0, int Q1>
__device__ __forceinline__ void bip_adj_chunk(const double *__restrict__ a1, const double *__restrict__ Ms,
                                              double *__restrict__ dM, const TgtInfo &ti, uint32_t tslot, int vrow,
                                              double o, int lane, double &ob) {
    constexpr int K = Q1 - Q0;
    double D[K], Mv[K], G[K];
    int cs[K];
#pragma unroll
    for (int u = 0; u < K; ++u) {
        const uint32_t sl = __shfl_sync(0xFFFFFFFFu, tslot, Q0 + u);
        const uint32_t meta = __shfl_sync(0xFFFFFFFFu, ti.meta, Q0 + u);
        cs[u] = (int)(((meta >> 12) & 15u) * 2u + ((meta >> 8) & 1u)) * kLanes;
        D[u] = a1[(size_t)sl * kLanes + lane];
        Mv[u] = Ms[vrow + cs[u]];
        G[u] = dM[vrow + cs[u]];
    }
#pragma unroll
    for (int u = 0; u < K; ++u) {
        ob = fma(D[u], Mv[u], ob);
        dM[vrow + cs[u]] = fma(D[u], o, G[u]);
    }
}

template <int NT>
__device__ __forceinline__ void bip_adj_endpoint(const double *fsrc, double *aout,
                                                 const double *__restrict__ a1, const double *__restrict__ Ms,
                                                 const double *__restrict__ Md, double *__restrict__ dM,
                                                 double *__restrict__ cdp, const TgtInfo &ti, uint32_t tslot,
                                                 uint32_t slot, int vrow, int hc, bool live, double cbar, double gamma,
                                                 int lane) {
    constexpr int kSplit = 6;
    // fsrc == aout: the forward state, replaced by its adjoint below (same slot, same thread)
    const double o = fsrc[(size_t)slot * kLanes + lane];
    double ob = 0.0;
    if constexpr (NT == 0) {
    } else if constexpr (NT <= kSplit) {
        bip_adj_chunk<0, NT>(a1, Ms, dM, ti, tslot, vrow, o, lane, ob);
    } else if constexpr (NT <= 2 * kSplit) {
        bip_adj_chunk<0, kSplit>(a1, Ms, dM, ti, tslot, vrow, o, lane, ob);
        bip_adj_chunk<kSplit, NT>(a1, Ms, dM, ti, tslot, vrow, o, lane, ob);
    } else {
        bip_adj_chunk<0, kSplit>(a1, Ms, dM, ti, tslot, vrow, o, lane, ob);
        bip_adj_chunk<kSplit, 2 * kSplit>(a1, Ms, dM, ti, tslot, vrow, o, lane, ob);
        bip_adj_chunk<2 * kSplit, NT>(a1, Ms, dM, ti, tslot, vrow, o, lane, ob);
    }
    // the close (a mask with a half-visited vertex, or a full mask); a dead mask closes into
    // nothing (warp-uniform test: no FP64 compare)
    if (live) {
        ob = fma(cbar, Md[vrow + hc], ob);
        *cdp = fma(gamma, o, *cdp);   // dM[(v,s)][(h,t)], or the closes' diagonal array when equal
    }
    aout[(size_t)slot * kLanes + lane] = ob;
}

__device__ __forceinline__ void bip_adj_dispatch(int nT, const double *fsrc, double *aout, const double *a1,
                                                 const double *Ms, const double *Md, double *dM, double *cdp,
                                                 const TgtInfo &ti, uint32_t tslot, uint32_t slot, int vrow, int hc,
                                                 bool live, double cbar, double gamma, int lane) {
#define COS_BADJ(K)                                                                                            \
    case K:                                                                                                    \
        bip_adj_endpoint<K>(fsrc, aout, a1, Ms, Md, dM, cdp, ti, tslot, slot, vrow, hc, live, cbar, gamma, lane); \
        break;
    switch (nT) {
        COS_BADJ(0)
        COS_BADJ(1)
        COS_BADJ(2)
        COS_BADJ(3)
        COS_BADJ(4)
        COS_BADJ(5)
        COS_BADJ(6)
        COS_BADJ(7)
        COS_BADJ(8)
        COS_BADJ(9)
        COS_BADJ(10)
        COS_BADJ(11)
        COS_BADJ(12)
        COS_BADJ(13)
        COS_BADJ(14)
        COS_BADJ(15)
        COS_BADJ(16)
        COS_BADJ(17)
        COS_BADJ(18)
        default:   // larger counts do not occur (at most 2 n - 1 targets, n <= COS_BIP_NMAX)
            break;
    }
#undef COS_BADJ
}

constexpr int kBipAdjMaxN = COS_BIP_NMAX;
// Largest order whose dM accumulators fit in shared memory beside Ms and Md (3 x 4 n^2 doubles
// per lane); above it dM lives in the CTA's global scratch, [(v,s)][(j,t)][lane] as in shared
// memory (coalesced per warp, mostly L1 / L2 resident).
constexpr int kBipAdjSmemMaxN = 8;

// UW: loop weight 1, so sgn w Cbar is a sign flip (no FP64 instruction).
template <bool CLOW, bool UW = true>
__global__ void __launch_bounds__(512, 1) dp_bip_adjoint_kernel(const __grid_constant__ BipAdjArgs a) {
    extern __shared__ __align__(16) double smem_ba[];
    __shared__ int s_batch;
    __shared__ uint32_t s_loc[2 * kBipAdjMaxN + 2];   // slot offset of each layer in the CTA's store
    // the batch's schedule: per step a layer, +256 for a forward step (the first pass over every
    // layer, then the refills of segments), else a reverse step
    __shared__ int s_ops[6 * kBipAdjMaxN + 2];
    __shared__ int s_nops;
    // the closes' diagonal terms dM[(h,t)][(h,t)], kept apart so that the diagonal of dM holds only
    // extension terms (their sum over v >= 1 per sublattice is dc/dsigma / sgn)
    __shared__ double s_dmd[2 * kBipAdjMaxN][kLanes];
    const BipArgs &f = a.f;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int nsm = 4 * f.smem_n * f.smem_n * kLanes;
    double *Ms = smem_ba;             // extension matrices (shifted diagonal)
    double *Md = smem_ba + nsm;       // close matrices times sgn w
    double *store = reinterpret_cast<double *>(f.scratch) + (size_t)blockIdx.x * a.cta_elems;
    // dc/dM accumulators [(v,s)][(j,t)][lane]
    double *dM = a.dm_global ? store + a.store_elems : smem_ba + 2 * nsm;
    const int nfl = f.nf_lanes;
    const int lam = lane % nfl;
    const int ci = lane / nfl;
    const double sgn = -1.0;
    double sig[2], seedsh[2];
    for (int s2 = 0; s2 < 2; ++s2) {
        sig[s2] = f.sigma2[lam][s2];
        seedsh[s2] = sgn * 2.0 * sig[s2];
    }
    const bool shifts = f.shifts != 0 && !CLOW;
    const double cfac = sgn * f.loop_weight;
    const int nbatch = *f.n_batches;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_batch = atomicAdd(f.queue, 1);
        __syncthreads();
        const int b = s_batch;
        if (b >= nbatch) break;
        const int4 bd = f.batches[b];
        const int n = bd.x;
        const int n2 = 2 * n;
        const BipOrderTab &tab = f.tabs[n];
        const bool active = (ci < bd.z) && (ci * nfl + nfl <= kLanes);
        const int cfg = active ? f.batch_list[bd.y + ci] : -1;
        const double *Mc = nullptr;
        if (active) Mc = f.M + f.moff[cfg] + (size_t)lam * n2 * n2;
        for (int e = warp; e < n2 * n2; e += nwarps) {
            const double val = active ? Mc[e] : 0.0;
            const int r = e / n2, c = e % n2;
            if (CLOW) {
                const double m = (r == c) ? val + sgn * sig[r & 1] : val;
                Ms[e * kLanes + lane] = m;
                Md[e * kLanes + lane] = cfac * m;
            } else {
                Ms[e * kLanes + lane] = ((r == c) && (r >= 2) && shifts) ? val + sgn * sig[r & 1] : val;
                Md[e * kLanes + lane] = cfac * val;
            }
            dM[e * kLanes + lane] = 0.0;
            if (r == c) s_dmd[r][lane] = 0.0;
        }
        if (threadIdx.x == 0) {
            // layer places: checkpoints (layer 1 and the plan's layers) back to back, then the
            // interior layers of one segment back to back after them
            const uint32_t ck = a.ckmask[n];
            uint32_t c = 0;
            int seg[2 * kBipAdjMaxN + 1], ns = 0;
            for (int l = 1; l <= 2 * n; ++l)
                if (l == 1 || ((ck >> l) & 1u)) {
                    s_loc[l] = c;
                    c += tab.layer_slots[l];
                    seg[ns++] = l;
                }
            uint32_t run = 0;
            for (int l = 2; l <= 2 * n; ++l) {
                if ((ck >> l) & 1u) {
                    run = 0;
                } else {
                    s_loc[l] = c + run;
                    run += tab.layer_slots[l];
                }
            }
            s_loc[2 * n + 1] = 0;   // the full masks extend nowhere: never written or read
            // the first forward pass, then the segments from the last: refill (all but the last),
            // then reverse its layers
            int no = 0;
            for (int ell = 1; ell <= 2 * n; ++ell) s_ops[no++] = ell + 256;
            for (int sg = ns - 1; sg >= 0; --sg) {
                const int lo = seg[sg], hi = (sg + 1 < ns) ? seg[sg + 1] : 2 * n + 1;
                if (sg + 1 < ns)
                    for (int ell = lo; ell <= hi - 2; ++ell) s_ops[no++] = ell + 256;
                for (int ell = hi - 1; ell >= lo; --ell) s_ops[no++] = ell;
            }
            s_nops = no;
        }
        __syncthreads();
        if (warp == 0) {
            for (int s0 = 0; s0 < 2; ++s0) {
                const uint32_t off = __ldg(tab.rank4 + 1 + s0);
                store[(size_t)(s_loc[1] + off + 3u * (uint32_t)s0) * kLanes + lane] = (CLOW && lam != 0) ? 0.0 : 1.0;
            }
        }
        __syncthreads();
        // the schedule: forward steps split masks over the warps; reverse steps take this warp's
        // endpoint units (v, s_v).  Only the batch's constants live across it: a reverse step
        // re-derives its own state, so the forward steps carry no register of the reverse sweep.
        for (int op = 0; op < s_nops; ++op) {
            const int step = s_ops[op];
            if (step >= 256) {
                // a forward step, every layer to its place: the first pass, or the refill of a
                // segment from its checkpoint (refills stop below layer 2n, so the sink is
                // written once, by the first pass)
                const int ell = step - 256;
                const double *src = store + (size_t)s_loc[ell] * kLanes;
                double *dst1 = store + (size_t)s_loc[ell + 1] * kLanes;
                const uint32_t first = tab.layer_first[ell], cnt = tab.layer_count[ell];
                for (uint32_t mi = warp; mi < cnt; mi += nwarps)
                    bip_mask<double, CLOW>(tab, first + mi, 0xFFFFFFFFu, ell, n, src, dst1, Ms, Md, lane, ci, nfl,
                                           seedsh, shifts, active, lam, cfg, f.out, f.status, 0);
                __syncthreads();
                continue;
            }
            const int ell = step;
            // own2 = this warp's units (v, s_v), own = the vertices with an owned unit
            uint32_t own2 = 0u, own = 0u;
            for (int u = warp; u < n2; u += nwarps) {
                own2 |= 1u << u;
                own |= 1u << (u >> 1);
            }
            const uint32_t full = (1u << n) - 1u;
            const double gout = active ? a.gout[cfg] : 0.0;
            const double cbar_full = CLOW ? gout : ldexp(gout, n - 1);   // Cbar of the full mask (the sink)
            double *aout = store + (size_t)s_loc[ell] * kLanes;   // O(ell), replaced by Obar(ell)
            const double *fsrc = aout;
            const double *a1 = store + (size_t)s_loc[ell + 1] * kLanes;
            const uint32_t first = tab.layer_first[ell], cnt = tab.layer_count[ell];
            for (uint32_t mi = 0; mi < cnt && own; ++mi) {
                const uint4 mk = __ldg(tab.masks + first + mi);
                const uint32_t A = mk.x & 0xFFFFu;
                if (!(A & own)) continue;
                const uint32_t B = mk.x >> 16, S = mk.y, code = mk.z, off = mk.w;
                const uint32_t ones = A & ~B;
                const uint32_t H = head_set(B, ones);
                const uint32_t J = full & ~B & (CLOW ? ~(ones & 1u) : 0xFFFFFFFFu);
                const int nA = __popc(A);
                const TgtInfo ti = bip_targets(A, B, S, J, code, tab.rank4, lane);
                const int nT = __popc(J) + __popc(J & ~A);
                const bool live = (ones != 0u) || (B == full);
                double cbar = 0.0;
                if (B == full) {
                    cbar = cbar_full;
                } else if (ones) {
                    const int k = __ffs(ones) - 1;
                    const uint32_t bk = 1u << k;
                    const int sk = (int)((S >> k) & 1u);
                    const uint32_t B1 = B | bk;
                    const uint32_t code1 = code + (uint32_t)(2 - sk) * c_p4[k];
                    const int hi1 = __popc(head_set(B1, A & ~B1) & (bk - 1u));
                    const uint32_t off1 = __ldg(tab.rank4 + code1);
                    const uint32_t ss = off1 + (uint32_t)(((hi1 * 2 + sk) * nA + __popc(A & (bk - 1u))) * 2 + sk);
                    const double seed = a1[(size_t)ss * kLanes + lane];
                    cbar = flavor_sum((CLOW && k == 0 && lam == 0) ? 0.0 : seed, nfl, ci);
                }
                const double gamma = UW ? neg(cbar) : cfac * cbar;
                for (uint32_t hh = H; hh; hh &= hh - 1u) {
                    const int h = __ffs(hh) - 1;
                    const int hidx = __popc(H & ((1u << h) - 1u));
                    const uint32_t Vrow = row_vmask(A, ones, h) & own;
                    if (!Vrow) continue;
                    const bool first_loop = (h == 0) && (ones & 1u);
                    const int sh0 = first_loop ? (int)(S & 1u) : 0;
                    const int sh1 = first_loop ? sh0 : 1;
                    const uint32_t hlow = (1u << h) - 1u;
                    const uint32_t ai1 = ti.meta & 15u, nA1 = (ti.meta >> 4) & 15u, sj1 = (ti.meta >> 8) & 1u;
                    const uint32_t hi1 = (uint32_t)__popc((ti.meta >> 16) & hlow);
                    for (int sh = sh0; sh <= sh1; ++sh) {
                        const uint32_t rowbase = off + (uint32_t)((hidx * 2 + sh) * nA * 2);
                        const uint32_t tslot = ti.off1 + ((hi1 * 2u + (uint32_t)sh) * nA1 + ai1) * 2u + sj1;
                        const int hc = (h * 2 + sh) * kLanes;
                        // the row's endpoint units 2v + s_v (the forward row's mask) that this warp
                        // owns, in ascending order
                        const uint32_t bh = 1u << h, vhalf = Vrow & ones;
                        uint32_t R = spread_even(Vrow & ~ones & ~bh) * 3u | spread_even(vhalf & ~S) |
                                     (spread_even(vhalf & S) << 1);
                        if (Vrow & ~ones & bh) R |= 1u << (2 * h + sh);
                        for (uint32_t rr = R & own2; rr; rr &= rr - 1u) {
                            const int u = __ffs(rr) - 1;
                            const uint32_t slot =
                                rowbase + (uint32_t)(__popc(A & ((1u << (u >> 1)) - 1u)) * 2 + (u & 1));
                            const int vrow = u * n2 * kLanes + lane;
                            double *cdp = (u == h * 2 + sh) ? &s_dmd[h * 2 + sh][lane] : dM + vrow + hc;
                            bip_adj_dispatch(nT, fsrc, aout, a1, Ms, Md, dM, cdp, ti, tslot, slot, vrow, hc, live,
                                             cbar, gamma, lane);
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (active && a.gM) {
            const int64_t gb = f.moff[cfg] + (int64_t)lam * n2 * n2;
            for (int e = warp; e < n2 * n2; e += nwarps) {
                const int r = e / n2;
                const double d = dM[e * kLanes + lane];
                a.gM[gb + e] = (r == e % n2) ? d + s_dmd[r][lane] : d;
            }
        }
        if (CLOW) {
            if (a.gsig && warp == 0 && active) {   // dc/dalpha_{b,s} = -sum_j dc/dM_b[(j,s)][(j,s)]
                double t0 = 0.0, t1 = 0.0;
                for (int j = 0; j < n; ++j) {
                    t0 += dM[((2 * j) * n2 + 2 * j) * kLanes + lane] + s_dmd[2 * j][lane];
                    t1 += dM[((2 * j + 1) * n2 + 2 * j + 1) * kLanes + lane] + s_dmd[2 * j + 1][lane];
                }
                a.gsig[((int64_t)cfg * nfl + lam) * 2] = -t0;
                a.gsig[((int64_t)cfg * nfl + lam) * 2 + 1] = -t1;
            }
        } else if (a.gsig) {
            if (warp == 0 && active) {
                // vertex 0's shifted start on sublattice s: sgn 2 times the adjoint of the seed slot
                // of its layer-1 mask's close, slot 3 s of the mask with vertex 0 full (code 3) in
                // layer 2, still in place
                const size_t sb = (size_t)s_loc[2] + __ldg(tab.rank4 + 3u);
                double t0 = sgn * 2.0 * store[sb * kLanes + lane];
                double t1 = sgn * 2.0 * store[(sb + 3u) * kLanes + lane];
                // the shifted diagonal (v >= 1): sgn times the extension part of dc/dM[(v,s)][(v,s)]
                for (int v = 1; v < n; ++v) {
                    t0 = fma(sgn, dM[((2 * v) * n2 + 2 * v) * kLanes + lane], t0);
                    t1 = fma(sgn, dM[((2 * v + 1) * n2 + 2 * v + 1) * kLanes + lane], t1);
                }
                a.gsig[((int64_t)cfg * nfl + lam) * 2] = t0;
                a.gsig[((int64_t)cfg * nfl + lam) * 2 + 1] = t1;
            }
        }
    }
}

static cos_status launch_bip_adjoint(Workspace *ws, const BipLaunch &L, const double *gout, double *gM,
                                     double *gsig, cudaStream_t stream) {
    std::string err;
    const BipOrderTab *tabs = bip_device_orders(ws->device, &err);
    if (!tabs) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    const bool dm_global = L.n_max > kBipAdjSmemMaxN;
    const size_t mat_elems = (size_t)4 * L.n_max * L.n_max * kLanes;
    const size_t extra = (dm_global ? mat_elems : 0) * sizeof(double);   // per CTA, beside the layers
    const int warps = std::min(16, std::max(4, 2 * L.n_max));
    const size_t smem = (dm_global ? 2 : 3) * mat_elems * sizeof(double);
    auto kern = L.clow ? dp_bip_adjoint_kernel<true>
                       : (L.loop_weight == 1 ? dp_bip_adjoint_kernel<false> : dp_bip_adjoint_kernel<false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "bipartite adjoint smem attribute");
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ws->device);
    const int cpb = kLanes / L.n_mat;
    const int max_batches = (L.n_cfg + cpb - 1) / cpb + COS_NMAX;
    const int gmax = std::max(1, std::min(nsm, max_batches));
    size_t free_b = 0, total_b = 0;
    size_t avail = (size_t)-1;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) avail = ws->scratch_bytes + (size_t)(0.85 * (double)free_b);
    auto slots_budget = [&](int g) -> uint64_t {
        const size_t per = avail / (size_t)g;
        return per > extra ? (per - extra) / (kLanes * sizeof(double)) : 1;
    };
    // grid and checkpoint plans: as the square adjoint (most CTAs per unit of work, in memory)
    const int mode = checkpoint_mode();
    const uint64_t fwd_work = ck_forward_work(COS_BIPARTITE, L.n_max);
    int grid = 1;
    uint64_t budget = 0;
    if (mode >= 0) {
        const CkPlan p = mode == 1 ? ck_plan(COS_BIPARTITE, L.n_max, 0) : ck_full(COS_BIPARTITE, L.n_max);
        if (mode == 0) budget = p.store;
        grid = (int)std::max<size_t>(1, std::min<size_t>((size_t)gmax, avail / (p.store * kLanes * 8 + extra)));
    } else {
        double best_score = -1.0;
        for (int g = gmax; g >= 1; g = (g > 8 ? g - std::max(1, g / 8) : g - 1)) {
            const uint64_t b = slots_budget(g);
            const CkPlan p = ck_plan(COS_BIPARTITE, L.n_max, b);
            if (!p.ok) continue;
            const double score = (double)g / (3.0 * (double)fwd_work + (double)p.recompute);
            if (score > best_score * (1.0 + 1e-9)) {
                best_score = score;
                grid = g;
                budget = b;
            }
        }
        if (best_score < 0) {
            grid = 1;
            budget = 0;
        }
    }
    uint32_t ckmask[COS_BIP_NMAX + 1] = {};
    uint64_t store_slots = 0;
    for (int n = 1; n <= L.n_max; ++n) {
        const CkPlan p = (mode == 0) ? ck_full(COS_BIPARTITE, n) : ck_plan(COS_BIPARTITE, n, budget);
        const CkPlan q = p.ok ? p : ck_plan(COS_BIPARTITE, n, 0);
        ckmask[n] = q.mask;
        store_slots = std::max(store_slots, q.store);
    }
    const size_t store_elems = (size_t)store_slots * kLanes;
    const size_t cta_elems = store_elems + (dm_global ? mat_elems : 0);
    ws->last_grid = grid;
    cos_status st = ensure(&ws->scratch, &ws->scratch_bytes, (size_t)grid * cta_elems * sizeof(double), 1,
                           "bipartite adjoint scratch");
    if (st != COS_OK) return st;
    BipAdjArgs a;
    memset(&a, 0, sizeof a);
    BipArgs &f = a.f;
    f.tabs = tabs;
    f.batches = ws->batches;
    f.n_batches = ws->plan_counts + 64;
    f.batch_list = ws->batch_list;
    f.queue = ws->queue;
    f.M = L.M;
    f.moff = L.moff;
    f.nf_lanes = L.n_mat;
    f.loop_weight = (double)L.loop_weight;
    memcpy(f.sigma2, L.sigma2, sizeof f.sigma2);
    f.shifts = L.shifts ? 1 : 0;
    f.scratch = ws->scratch;
    f.slot_elems = 0;
    f.smem_n = L.n_max;
    f.out = L.out;
    f.status = ws->status;
    a.store_elems = store_elems;
    a.cta_elems = cta_elems;
    memcpy(a.ckmask, ckmask, sizeof a.ckmask);
    a.gout = gout;
    a.gM = gM;
    a.gsig = gsig;
    a.dm_global = dm_global ? 1 : 0;
    e = cudaMemsetAsync(ws->queue, 0, sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e, "queue reset");
    kern<<<grid, warps * 32, smem, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "bipartite adjoint launch");
    return COS_OK;
}

static cos_status bip_grad_body(const char *fn, int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                                int n_mat, int loop_weight, const double *h_sigma2, const double *d_M4,
                                const double *d_gout, double *d_out, double *d_gM4, double *d_gsigma2, bool clow,
                                cudaStream_t stream) {
    cos_status st = check_bip(n_cfg, n_max, d_order, d_moff, n_mat, loop_weight, d_M4, COS_FP64, d_gout, fn);
    if (st != COS_OK) return st;
    if (n_cfg == 0) return COS_OK;
    std::string err;
    Workspace *ws = get_workspace(stream, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    BipLaunch L;
    L.precision = COS_FP64;
    L.clow = clow;
    L.n_cfg = n_cfg;
    L.n_max = n_max;
    L.order = d_order;
    L.M = d_M4;
    L.moff = d_moff;
    L.n_mat = n_mat;
    L.loop_weight = loop_weight;
    for (int l = 0; l < n_mat; ++l)
        for (int s2 = 0; s2 < 2; ++s2) {
            L.sigma2[l][s2] = h_sigma2 ? h_sigma2[l * 2 + s2] : 0.0;
            if (L.sigma2[l][s2] != 0.0) L.shifts = true;
        }
    L.out = d_out;
    st = launch_plan_batches(ws, n_cfg, n_max, d_order, kLanes / n_mat, stream);
    if (st != COS_OK) return st;
    return launch_bip_adjoint(ws, L, d_gout, d_gM4, d_gsigma2, stream);
}

cos_status bip_grad_dp(const char *fn, int n_cfg, int n_max, const int32_t *d_order, const int64_t *d_moff,
                       int n_mat, int loop_weight, const double *h_sigma2, const double *d_M4, const double *d_gout,
                       double *d_out, double *d_gM4, double *d_gsigma2, cudaStream_t stream, bool clow) {
    return bip_grad_body(fn, n_cfg, n_max, d_order, d_moff, n_mat, loop_weight, h_sigma2, d_M4, d_gout, d_out, d_gM4,
                         d_gsigma2, clow, stream);
}

}  // namespace cosdp

using namespace cosdp;

COS_INTERNAL_API cos_status cos_connected_sum_bipartite_matrices(int n_cfg, int n_max, const int32_t *d_order,
                                                           const int64_t *d_moff, int n_mat, int loop_weight,
                                                           const double *h_sigma2, const double *d_M4,
                                                           cos_precision precision, double *d_out,
                                                           double *d_abs_mass, cos_stream_t stream) {
    cos_status st = check_bip(n_cfg, n_max, d_order, d_moff, n_mat, loop_weight, d_M4, precision, d_out,
                              "cos_connected_sum_bipartite_matrices");
    if (st != COS_OK || n_cfg == 0) return st;
    std::string err;
    Workspace *ws = get_workspace((cudaStream_t)stream, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    return bip_matrices_body(ws, n_cfg, n_max, d_order, d_moff, n_mat, loop_weight, h_sigma2, d_M4, precision,
                             d_out, d_abs_mass, (cudaStream_t)stream, false);
}

COS_INTERNAL_API cos_status cos_connected_det_bipartite_matrices(int n_cfg, int n_max, const int32_t *d_order,
                                                           const int64_t *d_moff, const double *h_alpha2,
                                                           const double *d_M4, cos_precision precision,
                                                           double *d_out, double *d_abs_mass, cos_stream_t stream) {
    cos_status st = check_bip(n_cfg, n_max, d_order, d_moff, 2, 1, d_M4, precision, d_out,
                              "cos_connected_det_bipartite_matrices");
    if (st != COS_OK || n_cfg == 0) return st;
    std::string err;
    Workspace *ws = get_workspace((cudaStream_t)stream, &err);
    if (!ws) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    return bip_matrices_body(ws, n_cfg, n_max, d_order, d_moff, 2, 1, h_alpha2, d_M4, precision, d_out, d_abs_mass,
                             (cudaStream_t)stream, true);
}

extern "C" cos_status cos_bipartite_structure(int n, cos_structure_info *info) {
    if (n < 1 || n > COS_BIP_NMAX) {
        set_error("cos_bipartite_structure: order out of range");
        return COS_ERR_ORDER;
    }
    if (!info) {
        set_error("cos_bipartite_structure: null info");
        return COS_ERR_ARG;
    }
    *info = bip_host_order(n).info;
    return COS_OK;
}

COS_INTERNAL_API cos_status cos_connected_sum_bipartite_matrices_grad(int n_cfg, int n_max, const int32_t *d_order,
                                                                const int64_t *d_moff, int n_mat, int loop_weight,
                                                                const double *h_sigma2, const double *d_M4,
                                                                const double *d_gout, double *d_out, double *d_gM4,
                                                                double *d_gsigma2, cos_stream_t stream) {
    return bip_grad_body("cos_connected_sum_bipartite_matrices_grad", n_cfg, n_max, d_order, d_moff, n_mat,
                         loop_weight, h_sigma2, d_M4, d_gout, d_out, d_gM4, d_gsigma2, false, (cudaStream_t)stream);
}

COS_INTERNAL_API cos_status cos_connected_det_bipartite_matrices_grad(int n_cfg, int n_max, const int32_t *d_order,
                                                                const int64_t *d_moff, const double *h_alpha2,
                                                                const double *d_M4, const double *d_gout,
                                                                double *d_out, double *d_gM4, double *d_galpha2,
                                                                cos_stream_t stream) {
    return bip_grad_body("cos_connected_det_bipartite_matrices_grad", n_cfg, n_max, d_order, d_moff, 2, 1, h_alpha2,
                         d_M4, d_gout, d_out, d_gM4, d_galpha2, true, (cudaStream_t)stream);
}

namespace cosdp {
void bip_layer_profile(int n, uint64_t *slots, uint64_t *work) {
    const BipHostOrder &o = bip_host_order(n);
    for (int l = 0; l <= 2 * n; ++l) {
        slots[l] = o.layer_slots[l];
        work[l] = o.layer_work[l];
    }
}
}  // namespace cosdp
