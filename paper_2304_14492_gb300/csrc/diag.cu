// Diagnostics: the bounded-wait path of the tensor-core kernels, exercised on
// purpose.  k_wait_probe waits, with the same bounded mbarrier wait the MMA
// and copy pipelines use, on a barrier whose phase can never complete (two
// arrivals expected, one made), so the wait runs out after its time limit and
// the kernel reports ZM_ETIMEOUT in a status word and returns normally.
#include "tc_common.cuh"
#include "zm_internal.cuh"

namespace zm {

__global__ void k_wait_probe(int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = smem_u32(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;" ::"r"(b));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
    const bool done = mbar_wait(b, 0, global_ns());
    *status = done ? ZM_OK : ZM_ETIMEOUT;
}

}  // namespace zm

using namespace zm;

extern "C" int zm_probe_bounded_wait(int* status, void* stream) {
    if (!status) return set_error(ZM_EINVAL, "status is NULL");
    k_wait_probe<<<1, 32, 0, (cudaStream_t)stream>>>(status);
    ZM_LAUNCH_CHECK("k_wait_probe");
    return ZM_OK;
}
