// hd_noalloc.cu -- allocation-free batched convolution over a fixed work
// buffer that is part of the library image (see hd_convolve_batched_noalloc
// in include/hd.h for who needs it and the rules of use).
#include <cuda_runtime.h>

#include <mutex>

#include "hd_plan.h"

namespace {

// The fixed work buffer.  In host code this name is only a host-side handle of
// the device symbol; its device address is looked up per device below.
static __device__ __align__(256) unsigned char g_noalloc_work[HD_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices];

// Device address of g_noalloc_work on device `dev`, which must be current
// (looked up once per device).
hd_status work_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return HD_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_work) != cudaSuccess || !p) {
            cudaGetLastError();
            return HD_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return HD_OK;
}

}  // namespace

extern "C" hd_status hd_convolve_batched_noalloc(const hd_plan* plan, int64_t count, const void* const* f,
                                                  void* const* h, int64_t batch_stride, void* stream) {
    if (!plan || !f || !h || count < 0) return HD_ERR_INVALID;
    if (plan->ragged || plan->ndim != 1) return HD_ERR_INVALID;
    if (plan->sticky != HD_OK) return plan->sticky;
    const hd::AxisPlan& ax = plan->ax[0];
    if (ax.path != hd::PATH_SPLIT) return HD_ERR_UNSUPPORTED;
    for (int a = 0; a < plan->A; ++a)
        if (!f[a]) return HD_ERR_INVALID;
    for (int b = 0; b < plan->B; ++b)
        if (!h[b]) return HD_ERR_INVALID;
    if (count > 1 && batch_stride < plan->instance_elems) return HD_ERR_INVALID;
    const size_t esz = plan->dtype == HD_F64 ? 16 : 8;
    const size_t per = (size_t)(plan->A > plan->B ? plan->A : plan->B) * (size_t)hd::split_block(ax) * (size_t)ax.S * esz;
    if (per > HD_NOALLOC_SCRATCH_BYTES) return HD_ERR_SCRATCH_LIMIT;
    if (count == 0) return HD_OK;
    hd::DeviceGuard guard(plan->device);   // the plan's device, as hd_convolve_batched does
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    if (dev != plan->device) return HD_ERR_CUDA;
    void* work = nullptr;
    hd_status st = work_address(dev, &work);
    if (st != HD_OK) return st;
    const int64_t chunk = (int64_t)(HD_NOALLOC_SCRATCH_BYTES / per);
    st = hd::split_execute(*plan, ax, count, f, h, batch_stride, work, chunk, (cudaStream_t)stream);
    if (st == HD_ERR_CUDA) const_cast<hd_plan*>(plan)->sticky = st;
    return st;
}
