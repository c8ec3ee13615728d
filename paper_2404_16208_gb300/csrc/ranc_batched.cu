// Batched path (placeholder until the tensor-core kernel lands).
#include "ranc_internal.cuh"

namespace ranc {
cudaError_t batched_setup(ranc_sim *, const ranc_desc *, std::string &why) {
    why = "the batched path is not built in this version";
    return cudaErrorInvalidValue;
}
cudaError_t launch_batched_tick(ranc_sim *, const BatchedArgs &) { return cudaErrorNotSupported; }
cudaError_t launch_batched_reset(ranc_sim *, bool) { return cudaErrorNotSupported; }
cudaError_t launch_batched_inputs(ranc_sim *, const uint32_t *, int, int) { return cudaErrorNotSupported; }
cudaError_t launch_batched_export(ranc_sim *, int *, uint32_t *, uint32_t *) { return cudaErrorNotSupported; }
cudaError_t launch_batched_import(ranc_sim *, const int *, const uint32_t *) { return cudaErrorNotSupported; }
void batched_teardown(ranc_sim *) {}
}  // namespace ranc
