// Radial projection for callers that cannot allocate device memory.
//
// zm_project keeps its split-K partial sums in a workspace that the plan grows
// with cudaMalloc when a larger batch arrives.  Some callers cannot let the
// library allocate at call time: their device memory is already handed out by
// another allocator (a framework's caching pool that reserved the GPU up
// front), or they run in a loop where cudaMalloc's implicit device-wide
// synchronisation and unbounded latency are not acceptable.  zm_project_noalloc
// computes the same projection (the FP32 form, the kernels of zm_project's FP32
// path) with the partial sums in a fixed array in device memory that belongs to
// this file; it allocates nothing.  There is no counterpart in the paper: this
// is an interface matter only.
#include <mutex>

#include "zm_internal.cuh"

namespace zm {

// Fixed scratch: 2^21 floats (8 MiB).  Every GPU that loads this library's
// module holds it until the process exits.
constexpr size_t NOALLOC_FLOATS = (size_t)1 << 21;
static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_FLOATS];

// Device address of g_noalloc_scratch, looked up once per device with that
// device current (in host code the symbol itself is only a stand-in).  The
// address is kept for the life of the process: a device reset between calls
// (cudaDeviceReset, which reloads the module) is not supported.
static int noalloc_scratch(int dev, float** out) {
    static std::mutex mu;
    static float* addr[64] = {nullptr};
    if (dev < 0 || dev >= 64) return set_error(ZM_EUNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void* a = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-alloc scratch)");
        addr[dev] = static_cast<float*>(a);
    }
    *out = addr[dev];
    return ZM_OK;
}

}  // namespace zm

using namespace zm;

extern "C" int zm_project_noalloc(zm_plan_t plan, const float* spectra, int batch, float* out, unsigned flags,
                                  void* stream) {
    if (!plan || !spectra || !out) return set_error(ZM_EINVAL, "NULL argument");
    if (batch < 1) return set_error(ZM_EINVAL, "batch must be >= 1 (got %d)", batch);
    if (flags & ~ZM_NEUMANN) return set_error(ZM_EINVAL, "unknown flags 0x%x", flags);
    const size_t one_slice = (size_t)plan->P * 2 * batch;
    if (one_slice > NOALLOC_FLOATS)
        return set_error(ZM_EINVAL,
                         "zm_project_noalloc: P(n_max) * 2 * batch = %zu floats exceeds its fixed scratch of %zu "
                         "floats; use a smaller batch or zm_project",
                         one_slice, NOALLOC_FLOATS);
    DeviceGuard g(plan->device);
    if (!g.ok) return set_error(ZM_ECUDA, "cannot select device %d", plan->device);
    float* part = nullptr;
    const int s = noalloc_scratch(plan->device, &part);
    if (s != ZM_OK) return s;
    // the radial split is lowered until its slices fit the array
    return launch_projection_fp32_parts(plan, spectra, batch, out, flags, part, NOALLOC_FLOATS, (cudaStream_t)stream);
}
