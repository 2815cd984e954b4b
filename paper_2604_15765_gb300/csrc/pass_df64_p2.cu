// Instantiations of the fused pass kernels for the PolDF64 policy, tile
// sizes 3..5, 0..2 high qubits, for passes that contain a generic two-qubit map.
// One translation unit per policy and variant so they compile in parallel.
#include "pass_kernels.cuh"

namespace orkan {
cudaError_t launch_pass_df64_p2(void* state, const PassDesc& d, cudaStream_t s, int* launches) {
  return launch_p<PolDF64, true>(state, d, s, launches);
}
}  // namespace orkan
