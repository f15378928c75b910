// Mixed-precision step (FP32 pair gathers and sums, FP64 state): not built yet.
#include "tlsph_internal.cuh"

namespace tlsph {

cudaError_t launch_step_mixed(tlsph_ctx &, int64_t, cudaStream_t, cudaEvent_t *) { return cudaErrorNotSupported; }
cudaError_t mixed_sync_to_fp64(tlsph_ctx &, int, cudaStream_t) { return cudaSuccess; }
void mixed_release(tlsph_ctx &) {}

}  // namespace tlsph
