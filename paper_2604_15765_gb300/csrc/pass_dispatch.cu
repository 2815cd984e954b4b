// Pass launch dispatch by storage policy and by whether the pass holds a
// generic two-qubit map (whose kernels are compiled separately).
#include "orkan_internal.h"

namespace orkan {
cudaError_t launch_pass_f64(void* state, const PassDesc& d, cudaStream_t s, int* launches);
cudaError_t launch_pass_f32(void* state, const PassDesc& d, cudaStream_t s, int* launches);
cudaError_t launch_pass_df64(void* state, const PassDesc& d, cudaStream_t s, int* launches);
cudaError_t launch_pass_f64_p2(void* state, const PassDesc& d, cudaStream_t s, int* launches);
cudaError_t launch_pass_f32_p2(void* state, const PassDesc& d, cudaStream_t s, int* launches);
cudaError_t launch_pass_df64_p2(void* state, const PassDesc& d, cudaStream_t s, int* launches);

cudaError_t launch_pass(int dtype, void* state, const PassDesc& d, cudaStream_t s, int* launches) {
  if (launches) *launches = 0;
  switch (dtype) {
    case DT_C128: return d.has_ptm2 ? launch_pass_f64_p2(state, d, s, launches) : launch_pass_f64(state, d, s, launches);
    case DT_C64: return d.has_ptm2 ? launch_pass_f32_p2(state, d, s, launches) : launch_pass_f32(state, d, s, launches);
    case DT_DF64:
      return d.has_ptm2 ? launch_pass_df64_p2(state, d, s, launches) : launch_pass_df64(state, d, s, launches);
  }
  return cudaErrorInvalidValue;
}
}  // namespace orkan
