// Small device helpers shared by the pass and auxiliary kernels.
#pragma once
#include <cstdint>
#include "numeric.cuh"

namespace orkan {

// Row of the lower-triangular tile grid holding linear tile index g, i.e. the
// largest t with t (t + 1) / 2 <= g (tiles are stored row-major, Sec. III-B).
__device__ __forceinline__ int64_t tri_row(int64_t g) {
  int64_t t = (int64_t)((sqrtf((float)(8 * g + 1)) - 1.0f) * 0.5f);
  while (t > 0 && t * (t + 1) / 2 > g) --t;
  while ((t + 1) * (t + 2) / 2 <= g) ++t;
  return t;
}

__device__ __forceinline__ int64_t tile_base(int64_t ti, int64_t tj, int m) {
  return (ti * (ti + 1) / 2 + tj) << (2 * m);
}

// Element <-> FP64 complex conversions per storage policy.
template <class P> struct Conv;
template <> struct Conv<PolF64> {
  static __device__ __forceinline__ double2 to(double2 e) { return e; }
  static __device__ __forceinline__ double2 from(double re, double im) { return make_double2(re, im); }
};
template <> struct Conv<PolF32> {
  static __device__ __forceinline__ double2 to(float2 e) { return make_double2(e.x, e.y); }
  static __device__ __forceinline__ float2 from(double re, double im) { return make_float2((float)re, (float)im); }
};
template <> struct Conv<PolDF64> {
  // element order (re.hi, im.hi, re.lo, im.lo)
  static __device__ __forceinline__ double2 to(float4 e) {
    return make_double2((double)e.x + (double)e.z, (double)e.y + (double)e.w);
  }
  static __device__ __forceinline__ float4 from(double re, double im) {
    const float rh = __double2float_rn(re), ih = __double2float_rn(im);
    const float rl = __double2float_rn(re - (double)rh), il = __double2float_rn(im - (double)ih);
    return make_float4(rh, ih, rl, il);
  }
};

}  // namespace orkan
