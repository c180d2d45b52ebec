// Host-built structure of the merged clow-sequence DP for each order n.
//
// The interaction mask mu in {0,1,2}^n (Results A, contact-interaction merge) indexes
// the states; layer = number of visited points = sum_i mu_i.  Every configuration of
// one order shares this structure (the paper makes the same observation for its DAGs:
// the edge structure is configuration-independent, only matrix values differ), so it is
// built once on the host and kept on each device.
#include <algorithm>
#include <mutex>
#include <numeric>

#include "cos_internal.h"

namespace cosdp {

namespace {

int popc(uint32_t x) { return __builtin_popcount(x); }

void build_order(int n, HostOrder &o) {
    o.n = n;
    uint32_t p3[COS_NMAX + 2];
    p3[0] = 1;
    for (int i = 1; i <= n + 1; i++) p3[i] = 3 * p3[i - 1];
    const uint32_t full = (1u << n) - 1u;
    o.rank3.assign(p3[n], 0xFFFFFFFFu);
    o.ord3.assign(p3[n], 0xFFFFFFFFu);
    std::vector<std::vector<MaskRec>> per_layer(2 * n + 1);
    cos_structure_info &info = o.info;
    info = cos_structure_info{};
    info.n = n;
    for (uint32_t code = 0; code < p3[n]; code++) {
        uint32_t x = code, A = 0, B = 0;
        int layer = 0;
        for (int i = 0; i < n; i++) {
            uint32_t d = x % 3;
            x /= 3;
            if (d >= 1) A |= 1u << i;
            if (d == 2) B |= 1u << i;
            layer += (int)d;
        }
        if (!(A & 1u)) continue;
        const uint32_t ones = A & ~B;
        const uint32_t H = head_set(B, ones);
        const uint32_t J = full & ~B;
        const uint32_t Z = full & ~A;
        const bool needclose = ones != 0 || B == full;
        uint64_t cost = 0;
        for (uint32_t hh = H; hh; hh &= hh - 1) {
            int h = __builtin_ctz(hh);
            int nv = popc(row_vmask(A, ones, h));
            info.states += nv;
            info.fma_ext += (int64_t)nv * popc(J);
            if (needclose) info.fma_close += nv;
            info.mul_shift += popc(Z);
            cost += (uint64_t)nv * (popc(J) + (needclose ? 1 : 0)) + 4;
            o.layer_work[layer] += (uint64_t)nv * (popc(J) + (needclose ? 1 : 0));
        }
        MaskRec r;
        r.ab = A | (B << 16);
        r.code = code;
        r.off = 0;
        r.cost = (uint32_t)std::min<uint64_t>(cost, 0xFFFFFFFFu);
        per_layer[layer].push_back(r);
        info.masks++;
        info.slots += (int64_t)popc(H) * popc(A);
    }
    uint32_t first = 0;
    for (int l = 0; l <= 2 * n; l++) {
        auto &v = per_layer[l];
        std::stable_sort(v.begin(), v.end(), [](const MaskRec &a, const MaskRec &b) { return a.cost > b.cost; });
        uint32_t off = 0;
        uint32_t ordinal = 0;
        for (auto &r : v) {
            r.off = off;
            o.rank3[r.code] = off;
            o.ord3[r.code] = ordinal++;
            uint32_t A = r.ab & 0xFFFFu, B = r.ab >> 16;
            off += (uint32_t)(popc(head_set(B, A & ~B)) * popc(A));
        }
        o.layer_first[l] = first;
        o.layer_count[l] = (uint32_t)v.size();
        o.layer_slots[l] = off;
        o.max_slots = std::max(o.max_slots, off);
        o.max_masks = std::max(o.max_masks, (uint32_t)v.size());
        first += (uint32_t)v.size();
        o.masks.insert(o.masks.end(), v.begin(), v.end());
    }
    info.max_layer_slots = o.max_slots;
}

std::mutex g_mu;
HostOrder g_orders[COS_NMAX + 1];
bool g_built[COS_NMAX + 1];

struct DevOrders {
    OrderTab *d_tabs = nullptr;
};
DevOrders g_dev[64];

}  // namespace

const HostOrder &host_order(int n) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_built[n]) {
        build_order(n, g_orders[n]);
        g_built[n] = true;
    }
    return g_orders[n];
}

const OrderTab *device_orders(int device, std::string *err) {
    if (device < 0 || device >= 64) {
        *err = "device index out of range";
        return nullptr;
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_dev[device].d_tabs) return g_dev[device].d_tabs;
    }
    OrderTab tabs[COS_NMAX + 1];
    memset(tabs, 0, sizeof tabs);
    for (int n = 1; n <= COS_NMAX; n++) {
        const HostOrder &o = host_order(n);
        OrderTab &t = tabs[n];
        MaskRec *dm = nullptr;
        uint32_t *dr = nullptr, *dq = nullptr;
        cudaError_t e = cudaMalloc(&dm, o.masks.size() * sizeof(MaskRec));
        if (e == cudaSuccess) e = cudaMalloc(&dr, o.rank3.size() * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc(&dq, o.ord3.size() * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMemcpy(dm, o.masks.data(), o.masks.size() * sizeof(MaskRec), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dr, o.rank3.data(), o.rank3.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dq, o.ord3.data(), o.ord3.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            *err = std::string("structure upload: ") + cudaGetErrorString(e);
            return nullptr;
        }
        t.masks = dm;
        t.rank3 = dr;
        t.ord3 = dq;
        memcpy(t.layer_first, o.layer_first, sizeof t.layer_first);
        memcpy(t.layer_count, o.layer_count, sizeof t.layer_count);
        memcpy(t.layer_slots, o.layer_slots, sizeof t.layer_slots);
        t.max_slots = o.max_slots;
        t.max_masks = o.max_masks;
        t.n = n;
    }
    OrderTab *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof tabs);
    if (e == cudaSuccess) e = cudaMemcpy(d, tabs, sizeof tabs, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        *err = std::string("structure upload: ") + cudaGetErrorString(e);
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev[device].d_tabs) g_dev[device].d_tabs = d;
    return g_dev[device].d_tabs;
}

}  // namespace cosdp

extern "C" cos_status cos_structure(int n, cos_structure_info *info) {
    if (n < 1 || n > COS_NMAX) {
        cosdp::set_error("cos_structure: order out of range");
        return COS_ERR_ORDER;
    }
    if (!info) {
        cosdp::set_error("cos_structure: null info");
        return COS_ERR_ARG;
    }
    *info = cosdp::host_order(n).info;
    return COS_OK;
}
