// Connected sums from explicit matrices without any device allocation.
//
// Some callers cannot call cudaMalloc: code running inside a memory pool that owns the whole
// device, a host process that must not grow its footprint after start-up, or a plug-in that
// is handed a stream and buffers but no allocator.  For them this file keeps every scratch
// buffer of the DP -- planner tables, work queue, the per-order DP structure and the layer
// ring -- in one file-scope device array of fixed size.  This file is its own CUDA module
// (no kernels of its own), and under the runtime's lazy module loading (the default) that
// module -- and with it the 128 MiB array -- is loaded on a device by the first
// cudaGetSymbolAddress, i.e. during the first call of the entry point on that device.  From
// then on the device holds the array until the process exits.
//
// The array's name is only a host-side stand-in for the device symbol; its device address is
// obtained once per device with cudaGetSymbolAddress (with that device current) and passed to
// the kernels.  The first call on a device performs that set-up (module load, symbol address,
// copy of the DP structure tables); make that first call before a memory pool claims the
// device's free memory and before any stream capture.
//
// Kernels: the planner and the forward kernels of cos_dp.cu with one configuration per lane
// in every precision (FP64 dp_forward_kernel<double>, mixed <float>, double-float <df64>),
// not the two- and four-per-lane pair kernels the regular mixed and double-float calls use;
// warps per CTA come from the tuning line of (n_max, precision), which was measured for the
// regular call's kernel, so the mixed and double-float launch shapes here are untuned.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "cos_internal.h"

namespace cosdp {

namespace {

constexpr size_t kNoAllocBytes = size_t(128) << 20;  // 128 MiB
constexpr int kNoAllocNMax = 10;                      // largest order whose layers fit

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Fixed layout at the start of the array:
//   [0, 512)                 plan (80 ints), queue, status
//   [512, 512 + tabs bytes)  OrderTab[COS_NMAX + 1], then masks and rank3 of orders 1..kNoAllocNMax
//   [fixed_end, ...)         per call: batch list, batch table, layer ring
struct DevSetup {
    unsigned char *base = nullptr;
    size_t fixed_end = 0;
    bool ready = false;
};
std::mutex g_mu;
DevSetup g_setup[64];

cos_status setup_device(int dev, cudaStream_t stream, DevSetup **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    DevSetup &s = g_setup[dev];
    if (s.ready) {
        *out = &s;
        return COS_OK;
    }
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cos_connected_sum_matrices_noalloc: cudaGetSymbolAddress");
    unsigned char *base = static_cast<unsigned char *>(ptr);
    size_t off = 512;
    const size_t tabs_off = off;
    off = align256(off + sizeof(OrderTab) * (COS_NMAX + 1));
    OrderTab tabs[COS_NMAX + 1];
    memset(tabs, 0, sizeof tabs);
    for (int n = 1; n <= kNoAllocNMax; ++n) {
        const HostOrder &o = host_order(n);
        OrderTab &t = tabs[n];
        const size_t mbytes = o.masks.size() * sizeof(MaskRec), rbytes = o.rank3.size() * sizeof(uint32_t);
        e = cudaMemcpyAsync(base + off, o.masks.data(), mbytes, cudaMemcpyHostToDevice, stream);
        t.masks = reinterpret_cast<const MaskRec *>(base + off);
        off = align256(off + mbytes);
        if (e == cudaSuccess) e = cudaMemcpyAsync(base + off, o.rank3.data(), rbytes, cudaMemcpyHostToDevice, stream);
        t.rank3 = reinterpret_cast<const uint32_t *>(base + off);
        off = align256(off + rbytes);
        if (e != cudaSuccess) return cuda_fail(e, "cos_connected_sum_matrices_noalloc: structure copy");
        memcpy(t.layer_first, o.layer_first, sizeof t.layer_first);
        memcpy(t.layer_count, o.layer_count, sizeof t.layer_count);
        memcpy(t.layer_slots, o.layer_slots, sizeof t.layer_slots);
        t.max_slots = o.max_slots;
        t.max_masks = o.max_masks;
        t.ord3 = nullptr;   // used by the gradient only
        t.n = n;
    }
    e = cudaMemcpyAsync(base + tabs_off, tabs, sizeof tabs, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);   // host sources above are stack / cached vectors
    if (e != cudaSuccess) return cuda_fail(e, "cos_connected_sum_matrices_noalloc: structure copy");
    s.base = base;
    s.fixed_end = off;
    s.ready = true;
    *out = &s;
    return COS_OK;
}

}  // namespace

}  // namespace cosdp

using namespace cosdp;

extern "C" cos_status cos_connected_sum_matrices_noalloc(int n_cfg, int n_max, const int32_t *d_order,
                                                         const int64_t *d_moff, int n_mat, int loop_weight,
                                                         const double *h_sigma, const double *d_M,
                                                         cos_precision precision, double *d_out,
                                                         double *d_abs_mass, cos_stream_t stream) {
    const char *fn = "cos_connected_sum_matrices_noalloc";
    if (n_cfg < 0 || n_mat < 1 || n_mat > COS_MAX_FLAVORS || loop_weight < 1 ||
        (precision != COS_FP64 && precision != COS_MIXED && precision != COS_DF64)) {
        set_error(std::string(fn) + ": invalid argument");
        return COS_ERR_ARG;
    }
    if (n_max < 1 || n_max > kNoAllocNMax) {
        set_error(std::string(fn) + ": n_max outside [1, 10] (the fixed 128 MiB workspace holds the layers of "
                                    "orders up to 10)");
        return COS_ERR_ORDER;
    }
    if (n_cfg == 0) return COS_OK;
    if (!d_order || !d_moff || !d_M || !d_out) {
        set_error(std::string(fn) + ": null device pointer");
        return COS_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, fn);
    if (dev < 0 || dev >= 64) {
        set_error(std::string(fn) + ": device index out of range");
        return COS_ERR_ARG;
    }
    DevSetup *ds = nullptr;
    cos_status st = setup_device(dev, s, &ds);
    if (st != COS_OK) return st;

    DpLaunch L;
    L.n_cfg = n_cfg;
    L.n_max = n_max;
    L.order = d_order;
    L.M = d_M;
    L.moff = d_moff;
    L.n_mat = n_mat;
    L.loop_weight = loop_weight;
    for (int l = 0; l < n_mat; ++l) {
        L.sigma[l] = h_sigma ? h_sigma[l] : 0.0;
        if (L.sigma[l] != 0.0) L.shifts = true;
    }
    L.precision = precision;
    L.out = d_out;

    // Per-call layout after the fixed part; reject what does not fit.
    const int cpb = kLanes / n_mat;
    const size_t max_batches = (size_t)(n_cfg + cpb - 1) / cpb + COS_NMAX;
    size_t off = ds->fixed_end;
    const size_t list_off = off;
    off = align256(off + sizeof(int) * (size_t)n_cfg);
    const size_t batch_off = off;
    off = align256(off + sizeof(int4) * max_batches);
    const size_t per_cta = (size_t)dp_slots(L) * host_order(n_max).max_slots * kLanes * dp_state_bytes(L);
    if (off >= kNoAllocBytes || (kNoAllocBytes - off) / per_cta < 1) {
        set_error(std::string(fn) + ": batch too large for the fixed 128 MiB workspace (reduce n_cfg or n_max)");
        return COS_ERR_ARG;
    }
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const Tuning tu = get_tuning(n_max, precision, n_mat);
    const size_t fit = (kNoAllocBytes - off) / per_cta;
    int grid = (int)std::min<size_t>(fit, (size_t)nsm * tu.ctas_per_sm);
    grid = std::max(1, std::min<int>(grid, (int)max_batches));

    RawBuffers rb;
    rb.plan = reinterpret_cast<int *>(ds->base);
    rb.queue = rb.plan + 80;
    rb.status = rb.plan + 81;
    rb.list = reinterpret_cast<int *>(ds->base + list_off);
    rb.batches = reinterpret_cast<int4 *>(ds->base + batch_off);
    rb.scratch = ds->base + off;
    rb.tabs = reinterpret_cast<const OrderTab *>(ds->base + 512);
    rb.grid = grid;

    // Outputs start as NaN: a configuration whose order lies outside [1, n_max] is skipped by
    // the planner and keeps NaN (there is no status word to read back on this path).
    e = cudaMemsetAsync(d_out, 0xFF, sizeof(double) * (size_t)n_cfg, s);
    if (e == cudaSuccess && d_abs_mass) e = cudaMemsetAsync(d_abs_mass, 0xFF, sizeof(double) * (size_t)n_cfg, s);
    if (e != cudaSuccess) return cuda_fail(e, fn);
    st = launch_plan_raw(rb, n_cfg, n_max, d_order, cpb, dev, s);
    if (st != COS_OK) return st;
    st = launch_dp_raw(rb, L, s);
    if (st != COS_OK) return st;
    if (d_abs_mass) {
        L.out = d_abs_mass;
        L.absmode = true;
        st = launch_dp_raw(rb, L, s);
    }
    return st;
}
