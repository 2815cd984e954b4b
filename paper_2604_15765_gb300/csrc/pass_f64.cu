// Instantiations of the fused pass kernels for the PolF64 policy, tile
// sizes 3..5, 0..2 high qubits.
// One translation unit per policy and variant so they compile in parallel.
#include "pass_kernels.cuh"

namespace orkan {
cudaError_t launch_pass_f64(void* state, const PassDesc& d, cudaStream_t s, int* launches) {
  return launch_p<PolF64, false>(state, d, s, launches);
}
}  // namespace orkan
