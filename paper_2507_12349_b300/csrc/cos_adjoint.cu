// Reverse (adjoint) DP: gradient of every connected sum with respect to every propagator
// entry M^l[v][j] and to the shift weights sigma_l, then (tables path) by chain rule with
// respect to mu_l and alpha_l.
//
// For each batch the CTA first re-runs the forward sweep of cos_dp.cu (extension matrices
// with the shifted diagonal Ms[j][j] = M[j][j] - sigma, close matrices Mc = sgn w M), keeping
// every layer at exact per-layer offsets, then walks the layers backwards.  With Obar = dc/dO:
//   Cbar(full) = gout 2^(n-1);  Cbar(mu) = sum over the configuration's flavor lanes of
//   Obar(mu + e_k, k, k) when mu has a half-visited vertex (the seed it fed).
//   Row (mu, h), D_j = Obar(mu + e_j, h, j):
//     Obar(mu, h, v) = Cbar Mc[v][h] + sum_j D_j Ms[v][j]
//     dM[v][h] += sgn w Cbar O(mu,h,v);   dM[v][j] += D_j O(mu,h,v)   (dMs/dM = 1)
//     dsigma    = sgn sum over half-visited j >= 1 of D_j O(mu,h,j) (the shifted diagonal) +
//                 sgn 2 Obar(2e_0, 0, 0) (the shifted start); the first sum is the extension
//                 part of the diagonal of dM, read off once per batch (the closes' own diagonal
//                 terms accumulate apart, in dMd), the second read from layer 2 at the end.
// Every adjoint slot read was written earlier in the same sweep (targets of reachable edges
// are reachable), so nothing needs clearing.
//
// Storage.  Obar(mu,h,v) is formed by the one thread that reads O(mu,h,v), from that slot and
// the next layer's adjoints, and nothing reads O(mu,h,v) afterwards: the adjoint overwrites
// the forward state in place, so the reverse sweep needs no storage of its own.
// Checkpointing (memory-bound orders): the layers 1 = s_0 < s_1 < ... < s_m (checkpoints) are
// kept in a checkpoint area, the interior layers of one segment (s_i, s_{i+1}) in a segment
// area.  The first forward pass writes every layer to its place (a later segment overwrites an
// earlier one's interior); the reverse sweep then takes the segments from the last: for every
// segment but the last it re-runs the forward from its checkpoint to refill the segment area,
// then reverses its layers.  The plan (which layers are checkpoints) is chosen per order on the
// host to fit the CTAs' memory with the least recomputation (ck_plan below).
// Close adjoints: Cbar(mu) is a flavor sum of the seed slot's adjoints, formed once per mask by
// the warp that owns the seed slot (mu + e_k, k, k) when it computes that slot's adjoint, and
// left in a small plane of one value per (mask, lane) that the next layer's warps read.
// Determinant weights (CLOW instantiations, the sweep of Alg. 1 in cos_dp.cu): the forward
// recompute runs that mode, the reverse sweep skips the first loop's step onto vertex 0, a
// close at k = 0 fed block 1 only (Cbar = Obar of that lane), the sink's Cbar is gout, and the
// diagonal shifts sit in both matrix copies, so dc/dalpha_b = -sum_j dc/dM_b[j][j].
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>

#include "cos_dp_device.cuh"

namespace cosdp {

struct AdjArgs {
    DpArgs f;
    size_t store_elems;     // layer storage per CTA (checkpoint + segment areas) * 32
    size_t plane_elems;     // one close-adjoint plane: max masks per layer * 32
    size_t cta_elems;       // store_elems + 2 planes
    uint32_t ckmask[COS_NMAX + 1];   // per order: bit l = layer l is a checkpoint (0: every layer kept)
    const double *gout;
    double *gM;
    const int64_t *gmoff;
    int64_t gmstride;
    double *gsig;
};

// Reverse step of one endpoint v of row (mu, h), done by the warp that owns v, for a mask with
// NJ = |J| extensions (templated: every load is issued up front and no FP64 instruction is
// predicated off -- on B300 an FP64 instruction costs 16 SM cycles whether or not its lanes
// are enabled):
//   Obar(mu,h,v) = sum_j D_j Ms[v][j] + Cbar Mc[v][h],  dM[v][j] += D_j O,  dM[v][h] += gamma O.
// The close's own diagonal term (v = h) goes to dMd[h] instead of dM[h][h], so that dM[v][v]
// holds only the extension terms D_v O, whose sum over v >= 1 is dc/dsigma / sgn (the shifted
// diagonal): dsigma costs no multiply-add in the sweep.
// D_j = Obar(mu + e_j, h, j) is addressed through the mask's lane-parallel target table
// (mask_targets, shared with the forward push).  Cbar enters last, so its load overlaps the
// row's target loads.
// Extensions q in [Q0, Q1) of one endpoint: loads first, then the multiply-adds.
template <int Q0, int Q1>
__device__ __forceinline__ void adj_chunk(const double *__restrict__ a1, const double *__restrict__ Ms,
                                          double *__restrict__ dM, const TgtInfo &ti, uint32_t &jr, uint32_t hlow,
                                          int vrow, double o, int lane, double &ob) {
    constexpr int K = Q1 - Q0;
    double D[K], Mv[K], G[K];
    int js[K];
#pragma unroll
    for (int u = 0; u < K; ++u) {
        const uint32_t off1 = __shfl_sync(0xFFFFFFFFu, ti.off1, Q0 + u);
        const uint32_t meta = __shfl_sync(0xFFFFFFFFu, ti.meta, Q0 + u);
        const int j = __ffs(jr) - 1;
        jr &= jr - 1u;
        js[u] = j;
        const uint32_t ai1 = meta & 15u, nA1 = (meta >> 4) & 15u;
        const uint32_t hi1 = (uint32_t)__popc((meta >> 16) & hlow);
        D[u] = a1[(size_t)(off1 + hi1 * nA1 + ai1) * kLanes + lane];
        Mv[u] = Ms[vrow + j * kLanes];
        G[u] = dM[vrow + j * kLanes];
    }
#pragma unroll
    for (int u = 0; u < K; ++u) {
        ob = fma(D[u], Mv[u], ob);
        dM[vrow + js[u] * kLanes] = fma(D[u], o, G[u]);
    }
}

template <int NJ>
__device__ __forceinline__ double adj_endpoint(double *st, const double *__restrict__ a1,
                                               const double *__restrict__ Ms, const double *__restrict__ Mc,
                                               double *__restrict__ dM, double *__restrict__ dMd, const TgtInfo &ti,
                                               uint32_t J, int v, uint32_t slot, int h, int n, bool live,
                                               double cbar, double gamma, int lane) {
    constexpr int kSplit = 6;   // at most 6 extensions' operands in registers at a time
    // the forward state O(mu,h,v), replaced by its adjoint below (same slot, same thread)
    const double o = st[(size_t)slot * kLanes + lane];
    const int vrow = v * n * kLanes + lane;
    const uint32_t hlow = (1u << h) - 1u;
    uint32_t jr = J;
    double ob = 0.0;
    if constexpr (NJ == 0) {
        // full mask: the close into the sink only
    } else if constexpr (NJ <= kSplit) {
        adj_chunk<0, NJ>(a1, Ms, dM, ti, jr, hlow, vrow, o, lane, ob);
    } else {
        adj_chunk<0, kSplit>(a1, Ms, dM, ti, jr, hlow, vrow, o, lane, ob);
        adj_chunk<kSplit, NJ>(a1, Ms, dM, ti, jr, hlow, vrow, o, lane, ob);
    }
    // the close (a mask with a half-visited vertex, or the full mask); a dead mask closes into
    // nothing (warp-uniform test: no FP64 compare on the scarce pipe)
    if (live) {
        const int vh = vrow + h * kLanes;
        ob = fma(cbar, Mc[vh], ob);
        double *dp = (v == h) ? dMd + h * kLanes + lane : dM + vh;   // integer select of the address
        *dp = fma(gamma, o, *dp);
    }
    st[(size_t)slot * kLanes + lane] = ob;
    return ob;
}

// MAXNJ: the largest order the kernel instance runs (larger counts are never dispatched).
template <int MAXNJ>
__device__ __forceinline__ double adj_endpoint_dispatch(int nJ, double *st, const double *a1, const double *Ms,
                                                        const double *Mc, double *dM, double *dMd, const TgtInfo &ti,
                                                        uint32_t J, int v, uint32_t slot, int h, int n, bool live,
                                                        double cbar, double gamma, int lane) {
#define COS_AEP(K)                                                                                             \
    case K:                                                                                                    \
        if constexpr (K <= MAXNJ)                                                                              \
            return adj_endpoint<K>(st, a1, Ms, Mc, dM, dMd, ti, J, v, slot, h, n, live, cbar, gamma, lane);   \
        break;
    switch (nJ) {
        COS_AEP(0)
        COS_AEP(1)
        COS_AEP(2)
        COS_AEP(3)
        COS_AEP(4)
        COS_AEP(5)
        COS_AEP(6)
        COS_AEP(7)
        COS_AEP(8)
        COS_AEP(9)
        COS_AEP(10)
        COS_AEP(11)
        COS_AEP(12)
        default:
            break;
    }
#undef COS_AEP
    return 0.0;
}

// One layer of the forward sweep (masks split over the warps as in the forward kernel).
template <bool CLOW>
__device__ __forceinline__ void adj_forward_layer(const OrderTab &tab, int ell, int n, const double *src, double *dst1,
                                                  const double *Ms, const double *Mc, int lane, int warp, int nwarps,
                                                  int ci, int nfl, double sgn, double sig, bool shifts, bool active,
                                                  int lam, int cfg, double *out, int *status) {
    const uint32_t first = tab.layer_first[ell], cnt = tab.layer_count[ell];
    for (uint32_t mi = warp; mi < cnt; mi += nwarps)
        fwd_mask<double, false, CLOW>(tab, first + mi, mi + nwarps < cnt ? first + mi + nwarps : 0xFFFFFFFFu, ell, n,
                                      src, dst1, Ms, Mc, lane, ci, nfl, sgn, sig, shifts, active, lam, cfg, out,
                                      status, 1);
}

// Warps own endpoint vertices (v % warps == warp) in the reverse sweep, so the dM accumulators
// [v][j][lane] of the CTA have one writer per row v: one shared-memory copy, no atomics, each
// entry summed in a fixed order (bitwise reproducible).  Every warp walks every mask of a layer
// and takes the rows' endpoints it owns.  The forward passes split masks across warps as in the
// forward kernel.  MAXT = 320 (orders <= 10, two CTAs per SM) or 384 (one CTA).
// UW: loop weight 1, so sgn w Cbar is a sign flip (no FP64 instruction).
template <bool SG, int MAXT, bool CLOW = false, bool UW = true>
__global__ void __launch_bounds__(MAXT, MAXT <= 320 ? 2 : 1) dp_adjoint_kernel(const __grid_constant__ AdjArgs a) {
    extern __shared__ __align__(16) double smem_d[];
    __shared__ int s_batch;
    __shared__ uint32_t s_loc[kMaxLayers + 2];   // slot offset of each layer in the CTA's store
    __shared__ int s_seg[kMaxLayers + 1];        // segment starts: layer 1, then the checkpoints
    __shared__ int s_nseg;
    const DpArgs &f = a.f;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int nsm = f.smem_n * f.smem_n * kLanes;
    double *Ms = smem_d;              // extension matrices, shifted diagonal
    double *Mc = smem_d + nsm;        // close matrices times sgn w
    double *dM = smem_d + 2 * nsm;    // dc/dM accumulators [v][j][lane] (diagonal: extensions only)
    double *dMd = smem_d + 3 * nsm;   // the closes' diagonal terms [h][lane]
    double *store = reinterpret_cast<double *>(f.scratch) + (size_t)blockIdx.x * a.cta_elems;
    double *cplane = store + a.store_elems;   // two planes of close adjoints, by layer parity
    const int nfl = f.nf_lanes;
    const int lam = lane % nfl;
    const int ci = lane / nfl;
    const double sgn = -1.0;
    const double sig = f.sigma[lam];
    const bool shifts = f.shifts != 0;
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
        const OrderTab &tab = f.tabs[n];
        const bool active = (ci < bd.z) && (ci * nfl + nfl <= kLanes);
        const int cfg = active ? f.batch_list[bd.y + ci] : -1;
        const double *Mg = nullptr;
        if (active) Mg = f.M + (f.moff ? f.moff[cfg] : (int64_t)cfg * f.mstride) + (size_t)lam * n * n;
        for (int e = warp; e < n * n; e += nwarps) {
            const double val = active ? Mg[e] : 0.0;
            const int v = e / n, j = e % n;
            if (CLOW) {
                const double m = (v == j) ? val + sgn * sig : val;   // a(p, p) - alpha_b in both copies
                Ms[e * kLanes + lane] = m;
                Mc[e * kLanes + lane] = cfac * m;
            } else {
                Ms[e * kLanes + lane] = (v == j && j != 0 && shifts) ? val + sgn * sig : val;
                Mc[e * kLanes + lane] = cfac * val;
            }
            dM[e * kLanes + lane] = 0.0;
            if (v == j) dMd[v * kLanes + lane] = 0.0;
        }
        if (threadIdx.x == 0) {
            // layer places: checkpoints (layer 1 and the plan's layers) back to back, then the
            // interior layers of one segment back to back after them
            const uint32_t ck = a.ckmask[n];
            uint32_t c = 0;
            int ns = 0;
            for (int l = 1; l <= 2 * n; ++l)
                if (l == 1 || ((ck >> l) & 1u)) {
                    s_loc[l] = c;
                    c += tab.layer_slots[l];
                    s_seg[ns++] = l;
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
            s_loc[2 * n + 1] = 0;   // the full mask extends nowhere: never written or read
            s_nseg = ns;
        }
        __syncthreads();
        if (warp == 0) store[(size_t)s_loc[1] * kLanes + lane] = (CLOW && lam != 0) ? 0.0 : 1.0;
        __syncthreads();
        // first forward pass: every layer at its place
        for (int ell = 1; ell <= 2 * n; ++ell) {
            adj_forward_layer<CLOW>(tab, ell, n, store + (size_t)s_loc[ell] * kLanes,
                                    store + (size_t)s_loc[ell + 1] * kLanes, Ms, Mc, lane, warp, nwarps, ci, nfl, sgn,
                                    sig, shifts, active, lam, cfg, f.out, f.status);
            __syncthreads();
        }
        // reverse sweep, segment by segment from the last: this warp's endpoints
        uint32_t own = 0u;
        for (int v = warp; v < n; v += nwarps) own |= 1u << v;
        const uint32_t full = (1u << n) - 1u;
        const double gout = active ? a.gout[cfg] : 0.0;
        const double cbar_full = CLOW ? gout : ldexp(gout, n - 1);   // Cbar of the full mask (the sink)
        for (int sg = s_nseg - 1; sg >= 0; --sg) {
            const int lo = s_seg[sg], hi = (sg + 1 < s_nseg) ? s_seg[sg + 1] : 2 * n + 1;
            // refill the segment area from its checkpoint (the last segment is still in place)
            if (sg + 1 < s_nseg) {
                for (int ell = lo; ell <= hi - 2; ++ell) {
                    adj_forward_layer<CLOW>(tab, ell, n, store + (size_t)s_loc[ell] * kLanes,
                                            store + (size_t)s_loc[ell + 1] * kLanes, Ms, Mc, lane, warp, nwarps, ci,
                                            nfl, sgn, sig, shifts, active, lam, cfg, nullptr, f.status);
                    __syncthreads();
                }
            }
            for (int ell = hi - 1; ell >= lo; --ell) {
                double *st = store + (size_t)s_loc[ell] * kLanes;          // O(ell), replaced by Obar(ell)
                const double *a1 = store + (size_t)s_loc[ell + 1] * kLanes;  // Obar(ell + 1)
                const double *cin = cplane + (size_t)(ell & 1) * a.plane_elems;   // Cbar of this layer's masks
                double *cout = cplane + (size_t)((ell - 1) & 1) * a.plane_elems;  // Cbar of the layer below
                const uint32_t first = tab.layer_first[ell], cnt = tab.layer_count[ell];
                int turn = 2 % nwarps;   // (mi + 2) mod warps, kept by increments
                for (uint32_t mi = 0; mi < cnt && own; ++mi, turn = (turn + 1 == nwarps) ? 0 : turn + 1) {
                    const uint4 mk = __ldg(reinterpret_cast<const uint4 *>(tab.masks + first + mi));
                    // the warps take turns to pull a later mask's forward states into L2 ahead of use
                    if (mi + 2 < cnt && turn == warp) {
                        const uint4 nk = __ldg(reinterpret_cast<const uint4 *>(tab.masks + first + mi + 2));
                        const uint32_t nA_ = nk.x & 0xFFFFu, nB_ = nk.x >> 16;
                        prefetch_block(st, nk.z, (uint32_t)(__popc(head_set(nB_, nA_ & ~nB_)) * __popc(nA_)), lane,
                                       1);
                    }
                    const uint32_t A = mk.x & 0xFFFFu;
                    if (!(A & own)) continue;   // endpoints are visited vertices
                    const uint32_t B = mk.x >> 16, code = mk.y, off = mk.z;
                    const uint32_t ones = A & ~B;
                    const uint32_t H = head_set(B, ones);
                    const uint32_t J = full & ~B & (CLOW ? ~(ones & 1u) : 0xFFFFFFFFu);
                    const int nA = __popc(A);
                    const TgtInfo ti = mask_targets(A, B, J, code, tab.rank3, lane);
                    const int nJ = __popc(J);
                    const bool live = (ones != 0u) || (B == full);
                    double cbar = 0.0;
                    if (B == full) {
                        cbar = cbar_full;
                    } else if (ones) {
                        cbar = cin[(size_t)mi * kLanes + lane];   // flavor-summed by the seed slot's owner
                    }
                    const double gamma = UW ? neg(cbar) : cfac * cbar;
                    for (uint32_t hh = H; hh; hh &= hh - 1u) {
                        const int h = __ffs(hh) - 1;
                        const int hidx = __popc(H & ((1u << h) - 1u));
                        const uint32_t rowoff = off + (uint32_t)(hidx * nA);
                        for (uint32_t vv = row_vmask(A, ones, h) & own; vv; vv &= vv - 1u) {
                            const int v = __ffs(vv) - 1;
                            const uint32_t slot = rowoff + (uint32_t)__popc(A & ((1u << v) - 1u));
                            const double ob = adj_endpoint_dispatch<(MAXT <= 320 ? 10 : 12)>(
                                nJ, st, a1, Ms, Mc, dM, dMd, ti, J, v, slot, h, n, live, cbar, gamma, lane);
                            if (v == h && ((B >> h) & 1u)) {
                                // (mu, h, h) with h full is the seed slot of mu - e_h's close (the loop
                                // opened at h and has not moved): its flavor sum is that mask's Cbar
                                // (determinant weights: a close at k = 0 seeded block 1 only)
                                const double fs = flavor_sum((CLOW && h == 0 && lam == 0) ? 0.0 : ob, nfl, ci);
                                cout[(size_t)__ldg(tab.ord3 + code - c_p3[h]) * kLanes + lane] = fs;
                            }
                        }
                    }
                }
                __syncthreads();
            }
        }
        // dM rows are final (every warp passed the last barrier); dsigma: sum over warps in order
        if (active && a.gM) {
            const int64_t gb = (a.gmoff ? a.gmoff[cfg] : (int64_t)cfg * a.gmstride) + (int64_t)lam * n * n;
            for (int e = warp; e < n * n; e += nwarps) {
                const int v = e / n;
                const double d = dM[e * kLanes + lane];
                a.gM[gb + e] = (v == e % n) ? d + dMd[v * kLanes + lane] : d;
            }
        }
        if (CLOW && a.gsig) {   // dc/dalpha_b = -trace(dc/dM_b)
            if (warp == 0 && active) {
                double t = 0.0;
                for (int j = 0; j < n; ++j) t += dM[(j * n + j) * kLanes + lane] + dMd[j * kLanes + lane];
                a.gsig[(int64_t)cfg * nfl + lam] = -t;
            }
        } else if (SG) {
            // dsigma = sgn 2 Obar(2 e_0, 0, 0) (the shifted start: the seed slot of mask e_0's close,
            // mask code 1 + 3^0 in layer 2, still in place) + sgn sum_{v >= 1} (extension part of
            // dc/dM[v][v])
            if (warp == 0 && active && a.gsig) {
                double s = sgn * 2.0 * store[(size_t)(s_loc[2] + __ldg(tab.rank3 + 2u)) * kLanes + lane];
                for (int v = 1; v < n; ++v) s = fma(sgn, dM[(v * n + v) * kLanes + lane], s);
                a.gsig[(int64_t)cfg * nfl + lam] = s;
            }
        }
    }
}

// Chain rule through the tables: dc/dmu_l = sum_ij dc/dM^l_ij dM^l_ij/dmu_l, with dM/dmu the
// same linear interpolation of the dG/dmu table as the gather; dc/dalpha_l = -dc/dmu_l part
// + dc/dsigma_l / U.  Symmetric tables: the common derivative is split evenly over flavors.
__global__ void chain_kernel(const double *__restrict__ dG, int L, int n_tau, double beta, int n_mat, int n_flavors,
                             int symmetric, double U, int n_cfg, const int32_t *__restrict__ order,
                             const int64_t *__restrict__ offset, const int32_t *__restrict__ site,
                             const double *__restrict__ tau, const double *__restrict__ gM,
                             const int64_t *__restrict__ gmoff, int64_t gmstride, const double *__restrict__ gsig,
                             double *__restrict__ gmu, double *__restrict__ galpha) {
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int LL = L * L;
    const double scale = (double)(n_tau - 1) / beta;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_cfg; c += warps) {
        const int n = order[c];
        if (n < 1 || n > COS_NMAX || (!gmoff && (int64_t)n_mat * n * n > gmstride)) continue;
        const int64_t o = offset[c];
        const double *g = gM + (gmoff ? gmoff[c] : (int64_t)c * gmstride);
        for (int l = 0; l < n_mat; ++l) {
            double acc = 0.0;
            for (int e = lane; e < n * n; e += 32) {
                const int i = e / n, j = e % n;
                const int si = site[o + i], sj = site[o + j];
                if (si < 0 || si >= LL || sj < 0 || sj >= LL) continue;
                const int dx = ((si % L) - (sj % L) + L) % L;
                const int dy = ((si / L) - (sj / L) + L) % L;
                const double dt = tau[o + i] - tau[o + j];
                double s = 1.0, tt = dt;
                if (dt <= 0.0) {
                    s = -1.0;
                    tt = dt + beta;
                }
                const double x = tt * scale;
                int m = (int)floor(x);
                m = max(0, min(m, n_tau - 2));
                const double fr = x - m;
                const double *row = dG + ((size_t)l * LL + dx + L * dy) * n_tau + m;
                acc = fma(g[(size_t)l * n * n + e], s * fma(fr, row[1] - row[0], row[0]), acc);
            }
            for (int w = 16; w >= 1; w >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, w);
            if (lane == 0) {
                if (symmetric) {
                    for (int q = 0; q < n_flavors; ++q) {
                        const double dmu = acc / n_flavors;
                        if (gmu) gmu[(int64_t)c * n_flavors + q] = dmu;
                        if (galpha) galpha[(int64_t)c * n_flavors + q] = -dmu + gsig[c] / (n_flavors * U);
                    }
                } else {
                    if (gmu) gmu[(int64_t)c * n_flavors + l] = acc;
                    if (galpha) galpha[(int64_t)c * n_flavors + l] = -acc + gsig[(int64_t)c * n_mat + l] / U;
                }
            }
        }
    }
}

// Warps per adjoint CTA: one per vertex of the largest order (at least 4), so each warp owns one
// endpoint in the reverse sweep.
int adjoint_warps(int n_max) { return std::max(4, std::min(12, n_max)); }

// ------------------------------------------------------------------ checkpoint plans
//
// Storage (state slots per lane) and recomputation (multiply-adds of one flavor array) of a set
// of checkpoint layers, in the layout of the adjoint kernels: layer 1 and the checkpoints back
// to back, then room for the largest segment interior.  A segment other than the last is re-run
// from its checkpoint: the forward steps out of its layers s_i .. s_{i+1} - 2.

// Per-layer slots and sweep work of an order (square lattice: the merged structure; bipartite:
// the sublattice-resolved one).
struct LayerProfile {
    int n = 0;
    uint64_t slots[kMaxLayers + 1] = {};
    uint64_t work[kMaxLayers + 1] = {};
};

static LayerProfile layer_profile(int lattice, int n) {
    LayerProfile p;
    p.n = n;
    if (lattice == COS_BIPARTITE) {
        bip_layer_profile(n, p.slots, p.work);
    } else {
        const HostOrder &o = host_order(n);
        for (int l = 0; l <= 2 * n; ++l) {
            p.slots[l] = o.layer_slots[l];
            p.work[l] = o.layer_work[l];
        }
    }
    return p;
}

static CkPlan ck_eval(const LayerProfile &o, uint32_t mask) {
    const int L = 2 * o.n;
    uint64_t ck = o.slots[1], interior = 0, segmax = 0, rec = 0;
    int start = 1;
    for (int l = 2; l <= L; ++l) {
        if ((mask >> l) & 1u) {
            segmax = std::max(segmax, interior);
            for (int e = start; e <= l - 2; ++e) rec += o.work[e];
            start = l;
            interior = 0;
            ck += o.slots[l];
        } else {
            interior += o.slots[l];
        }
    }
    segmax = std::max(segmax, interior);
    CkPlan p;
    p.mask = mask;
    p.store = ck + segmax;
    p.recompute = rec;
    p.ok = true;
    return p;
}

constexpr int kMaxCheckpoints = 7;   // enough for the optimum at every order up to 12

// Pareto frontier of the checkpoint sets of an order (every set of at most kMaxCheckpoints layers
// among 2 .. 2n, and the empty set): increasing storage, strictly decreasing recomputation.  The
// first point needs the least storage; the last is the empty set (no recomputation).
static const std::vector<CkPlan> &ck_frontier(int lattice, int n) {
    static std::mutex mu;
    static std::vector<CkPlan> cache[2][COS_NMAX + 1];
    std::lock_guard<std::mutex> lk(mu);
    std::vector<CkPlan> &fr = cache[lattice == COS_BIPARTITE ? 1 : 0][n];
    if (!fr.empty()) return fr;
    const LayerProfile o = layer_profile(lattice, n);
    std::vector<CkPlan> all;
    all.push_back(ck_eval(o, 0u));
    struct Rec {
        const LayerProfile &o;
        int L;
        std::vector<CkPlan> &all;
        void go(int from, int k, uint32_t mask) {
            for (int l = from; l <= L; ++l) {
                const uint32_t m = mask | (1u << l);
                all.push_back(ck_eval(o, m));
                if (k + 1 < kMaxCheckpoints) go(l + 1, k + 1, m);
            }
        }
    } rec{o, 2 * n, all};
    rec.go(2, 0, 0u);
    std::sort(all.begin(), all.end(), [](const CkPlan &a, const CkPlan &b) {
        return a.store != b.store ? a.store < b.store
               : a.recompute != b.recompute ? a.recompute < b.recompute : a.mask < b.mask;
    });
    for (const CkPlan &c : all)
        if (fr.empty() || c.recompute < fr.back().recompute) fr.push_back(c);
    return fr;
}

CkPlan ck_plan(int lattice, int n, uint64_t budget) {
    const std::vector<CkPlan> &fr = ck_frontier(lattice, n);
    if (budget == 0) return fr.front();
    CkPlan best;
    for (const CkPlan &c : fr)
        if (c.store <= budget) best = c;   // recomputation decreases along the frontier
    return best;
}

CkPlan ck_full(int lattice, int n) { return ck_frontier(lattice, n).back(); }

uint64_t ck_forward_work(int lattice, int n) {
    const LayerProfile o = layer_profile(lattice, n);
    uint64_t w = 0;
    for (int l = 1; l <= 2 * n; ++l) w += o.work[l];
    return w;
}

// COS_GRAD_CHECKPOINT=1: every order keeps the least storage (recomputing the most); =0: every
// layer kept whatever the memory; unset: the plan that gives the most throughput within memory.
int checkpoint_mode() {
    const char *e = getenv("COS_GRAD_CHECKPOINT");
    if (!e || !*e) return -1;
    return e[0] == '0' ? 0 : 1;
}

cos_status launch_adjoint(Workspace *ws, const DpLaunch &L, const double *gout, double *gM, const int64_t *gmoff,
                          int64_t gmstride, double *gsig, cudaStream_t stream) {
    std::string err;
    const OrderTab *tabs = device_orders(ws->device, &err);
    if (!tabs) {
        set_error(err);
        return COS_ERR_CUDA;
    }
    const int n_max = L.n_max;
    const HostOrder &ho = host_order(n_max);
    const size_t plane_elems = (size_t)ho.max_masks * kLanes;
    const int warps = adjoint_warps(n_max);
    const int threads = warps * 32;
    const size_t smem = ((size_t)3 * n_max * n_max + n_max) * kLanes * sizeof(double);
    const bool sg = gsig != nullptr;
    const bool big = threads > 320;
    const bool uw = L.loop_weight == 1;
    auto kern = L.clow ? (big ? dp_adjoint_kernel<false, 384, true> : dp_adjoint_kernel<false, 320, true>)
                : uw   ? (sg ? (big ? dp_adjoint_kernel<true, 384> : dp_adjoint_kernel<true, 320>)
                             : (big ? dp_adjoint_kernel<false, 384> : dp_adjoint_kernel<false, 320>))
                       : (sg ? (big ? dp_adjoint_kernel<true, 384, false, false> : dp_adjoint_kernel<true, 320, false, false>)
                             : (big ? dp_adjoint_kernel<false, 384, false, false>
                                    : dp_adjoint_kernel<false, 320, false, false>));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint smem attribute");
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ws->device);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int cpb = kLanes / L.n_mat;
    const int max_batches = (L.n_cfg + cpb - 1) / cpb + COS_NMAX;
    const int gmax = std::max(1, std::min(nsm * std::min(per_sm, 2), max_batches));
    size_t free_b = 0, total_b = 0;
    size_t avail = (size_t)-1;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) avail = ws->scratch_bytes + (size_t)(0.85 * (double)free_b);
    const size_t plane_bytes = 2 * plane_elems * sizeof(double);
    auto slots_budget = [&](int g) -> uint64_t {
        const size_t per = avail / (size_t)g;
        return per > plane_bytes ? (per - plane_bytes) / (kLanes * sizeof(double)) : 1;
    };
    // Grid and checkpoint plan of the largest order: the most throughput, CTAs x the inverse of
    // the work per batch (forward, reverse = 2 forwards, and the recomputed segments).
    const int mode = checkpoint_mode();
    const uint64_t fwd_work = ck_forward_work(COS_SQUARE, n_max);
    int grid = 1;
    uint64_t budget = 0;   // slots per lane of every order's plan (0: least storage)
    if (mode == 1) {
        const CkPlan p = ck_plan(COS_SQUARE, n_max, 0);
        grid = (int)std::max<size_t>(1, std::min<size_t>((size_t)gmax, avail / (p.store * kLanes * 8 + plane_bytes)));
    } else if (mode == 0) {
        const CkPlan p = ck_full(COS_SQUARE, n_max);
        budget = p.store;
        grid = (int)std::max<size_t>(1, std::min<size_t>((size_t)gmax, avail / (p.store * kLanes * 8 + plane_bytes)));
    } else {
        double best_score = -1.0;
        for (int g = gmax; g >= 1; g = (g > 8 ? g - std::max(1, g / 8) : g - 1)) {
            const uint64_t b = slots_budget(g);
            const CkPlan p = ck_plan(COS_SQUARE, n_max, b);
            if (!p.ok) continue;
            const double score = (double)g / (3.0 * (double)fwd_work + (double)p.recompute);
            if (score > best_score * (1.0 + 1e-9)) {
                best_score = score;
                grid = g;
                budget = b;
            }
        }
        if (best_score < 0) {   // not even one CTA fits: least storage, one CTA
            grid = 1;
            budget = 0;
        }
    }
    AdjArgs a;
    memset(&a, 0, sizeof a);
    uint64_t store_slots = 0;
    for (int n = 1; n <= n_max; ++n) {
        const CkPlan p = (mode == 0) ? ck_full(COS_SQUARE, n) : ck_plan(COS_SQUARE, n, budget);
        const CkPlan q = p.ok ? p : ck_plan(COS_SQUARE, n, 0);
        a.ckmask[n] = q.mask;
        store_slots = std::max(store_slots, q.store);
    }
    const size_t store_elems = (size_t)store_slots * kLanes;
    const size_t cta_elems = store_elems + 2 * plane_elems;
    cos_status st = ensure(&ws->scratch, &ws->scratch_bytes, (size_t)grid * cta_elems * sizeof(double), 1,
                           "adjoint scratch");
    if (st != COS_OK) return st;
    DpArgs &f = a.f;
    f.tabs = tabs;
    f.batches = ws->batches;
    f.n_batches = ws->plan_counts + 64;
    f.batch_list = ws->batch_list;
    f.queue = ws->queue;
    f.M = L.M;
    f.moff = L.moff;
    f.mstride = L.mstride;
    f.nf_lanes = L.n_mat;
    f.loop_weight = (double)L.loop_weight;
    for (int l = 0; l < COS_MAX_FLAVORS; ++l) f.sigma[l] = L.sigma[l];
    f.shifts = L.shifts ? 1 : 0;
    f.absmode = 0;
    f.scratch = ws->scratch;
    f.slot_elems = 0;
    f.nslots = 0;
    f.smem_n = n_max;
    f.out = L.out;
    f.status = ws->status;
    a.store_elems = store_elems;
    a.plane_elems = plane_elems;
    a.cta_elems = cta_elems;
    a.gout = gout;
    a.gM = gM;
    a.gmoff = gmoff;
    a.gmstride = gmstride;
    a.gsig = gsig;
    ws->last_grid = grid;
    e = cudaMemsetAsync(ws->queue, 0, sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e, "queue reset");
    kern<<<grid, warps * 32, smem, stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "adjoint launch");
    return COS_OK;
}

cos_status launch_chain(const cos_tables *t, int n_cfg, const int32_t *order, const int64_t *offset,
                        const int32_t *site, const double *tau, const double *gM, const int64_t *gmoff,
                        int64_t gmstride, const double *gsig, double *gmu, double *galpha, cudaStream_t stream) {
    if (n_cfg == 0) return COS_OK;
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, t->device);
    const int threads = 256;
    const int blocks = std::max(1, std::min((n_cfg * 32 + threads - 1) / threads, 8 * nsm));
    chain_kernel<<<blocks, threads, 0, stream>>>(t->d_dG, t->model.L, t->model.n_tau, t->model.beta, t->n_mat,
                                                  t->model.n_flavors, t->symmetric, t->model.U, n_cfg, order, offset,
                                                  site, tau, gM, gmoff, gmstride, gsig, gmu, galpha);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "chain launch");
    return COS_OK;
}

}  // namespace cosdp

extern "C" cos_status cos_grad_checkpoint_plan(int n, int64_t slots_budget, uint32_t *ck_mask, int64_t *store_slots,
                                               int64_t *recompute_fma) {
    if (n < 1 || n > COS_NMAX) {
        cosdp::set_error("cos_grad_checkpoint_plan: order out of range");
        return COS_ERR_ORDER;
    }
    if (slots_budget < 0 || !ck_mask || !store_slots || !recompute_fma) {
        cosdp::set_error("cos_grad_checkpoint_plan: invalid argument");
        return COS_ERR_ARG;
    }
    const cosdp::CkPlan p = cosdp::ck_plan(COS_SQUARE, n, (uint64_t)slots_budget);
    if (!p.ok) {
        cosdp::set_error("cos_grad_checkpoint_plan: no checkpoint plan fits the budget");
        return COS_ERR_ARG;
    }
    *ck_mask = p.mask;
    *store_slots = (int64_t)p.store;
    *recompute_fma = (int64_t)p.recompute;
    return COS_OK;
}
