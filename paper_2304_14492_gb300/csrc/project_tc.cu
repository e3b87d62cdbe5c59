// Radial projection on the tensor cores (bf16 / fp16 hi+lo split, FP32
// accumulate).
#include "zm_internal.cuh"

namespace zm {

int launch_projection_tc(zm_plan_t p, const float* F, int batch, float* out, unsigned flags, cudaStream_t st) {
    (void)p; (void)F; (void)batch; (void)out; (void)flags; (void)st;
    return set_error(ZM_EUNSUPPORTED, "tensor-core projection is not built yet");
}

}  // namespace zm
