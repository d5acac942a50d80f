// grpic_push32.cu -- FP32 form of the push + deposit (placeholder until the
// FP32 kernel lands).
#include "grpic_internal.cuh"

namespace grpic {
cudaError_t launch_push32(grpic_ctx *, grpic_particles *, grpic_fields *, bool, cudaStream_t)
{
    return cudaErrorNotSupported;
}
}  // namespace grpic
