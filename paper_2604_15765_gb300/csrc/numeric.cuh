// Arithmetic policies of the pass kernels.
//
//   PolF64  : complex128 storage, native FP64 arithmetic.
//   PolF32  : complex64 storage, FP32 arithmetic.
//   PolDF64 : 16-byte "double-float" storage (hi + lo float pairs for the real
//             and imaginary parts) and FP32-pipe arithmetic built from the
//             error-free transformations TwoSum (Knuth, TAOCP vol. 2) and
//             TwoProduct via FMA (Ogita, Rump, Oishi, SIAM J. Sci. Comput. 26,
//             2005), following the double-float format of Dekker (Numer.
//             Math. 18, 1971).  About 48 significand bits.
//
// GB300 runs FP64 at ~1/64 of the FP32 rate, so only the FP32 pipe can keep a
// conjugation pass at HBM speed; PolDF64 trades 5 bits of precision for that.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace orkan {

// ------------------------------------------------------------------ FP64
struct PolF64 {
  using Elem = double2;
  using Real = double;
  using Coef = double;
  static constexpr int kSwizzle = 7;  // 16-byte elements: 8 per 128-byte bank line
  static constexpr int kSwShift = 0;  // swizzle granule = 1 element (16 B)
  static __device__ __forceinline__ Coef coef(const double* c, int i) { return c[i]; }
  // conjugate when t == 1, by flipping the sign bit (no FP64 instruction)
  static __device__ __forceinline__ Elem conj_if(Elem e, unsigned t) {
    e.y = __hiloint2double(__double2hiint(e.y) ^ int(t << 31), __double2loint(e.y));
    return e;
  }
  static __device__ __forceinline__ Real re(const Elem& e) { return e.x; }
  static __device__ __forceinline__ Real im(const Elem& e) { return e.y; }
  static __device__ __forceinline__ Elem make(Real r, Real i) { return make_double2(r, i); }
  static __device__ __forceinline__ Elem conj(Elem e) { e.y = -e.y; return e; }
  static __device__ __forceinline__ Real add(Real a, Real b) { return a + b; }
  static __device__ __forceinline__ Real sub(Real a, Real b) { return a - b; }
  static __device__ __forceinline__ Real neg(Real a) { return -a; }
  // -a by flipping the sign bit with integer ops (no FP64 pipe instruction)
  static __device__ __forceinline__ Real flip(Real a) {
    return __hiloint2double(__double2hiint(a) ^ int(0x80000000u), __double2loint(a));
  }
  static __device__ __forceinline__ Real half(Real a) { return 0.5 * a; }
  static __device__ __forceinline__ Real mul(Real x, Coef c) { return x * c; }
  static __device__ __forceinline__ Real mac(Real acc, Real x, Coef c) { return fma(x, c, acc); }
  static __device__ __forceinline__ Real norm(Real a) { return a; }
  static __device__ __forceinline__ double to_double(Real a) { return a; }
};

// ------------------------------------------------------------------ FP32
struct PolF32 {
  using Elem = float2;
  using Real = float;
  using Coef = float;
  static constexpr int kSwizzle = 15;  // 8-byte elements: 16 per 128-byte bank line
  static constexpr int kSwShift = 1;   // swizzle granule = 2 elements (16 B, one cp.async)
  static __device__ __forceinline__ Coef coef(const double* c, int i) {
    return reinterpret_cast<const float*>(c)[2 * i];
  }
  static __device__ __forceinline__ Elem conj_if(Elem e, unsigned t) {
    e.y = __int_as_float(__float_as_int(e.y) ^ int(t << 31));
    return e;
  }
  static __device__ __forceinline__ Real re(const Elem& e) { return e.x; }
  static __device__ __forceinline__ Real im(const Elem& e) { return e.y; }
  static __device__ __forceinline__ Elem make(Real r, Real i) { return make_float2(r, i); }
  static __device__ __forceinline__ Elem conj(Elem e) { e.y = -e.y; return e; }
  static __device__ __forceinline__ Real add(Real a, Real b) { return a + b; }
  static __device__ __forceinline__ Real sub(Real a, Real b) { return a - b; }
  static __device__ __forceinline__ Real neg(Real a) { return -a; }
  static __device__ __forceinline__ Real flip(Real a) { return __int_as_float(__float_as_int(a) ^ int(0x80000000u)); }
  static __device__ __forceinline__ Real half(Real a) { return 0.5f * a; }
  static __device__ __forceinline__ Real mul(Real x, Coef c) { return x * c; }
  static __device__ __forceinline__ Real mac(Real acc, Real x, Coef c) { return fmaf(x, c, acc); }
  static __device__ __forceinline__ Real norm(Real a) { return a; }
  static __device__ __forceinline__ double to_double(Real a) { return (double)a; }
};

// ------------------------------------------------------------------ double-float
struct DF {
  float hi, lo;
};

// TwoSum: s + e == a + b exactly (no ordering assumption).  The _rn
// intrinsics keep the compiler from contracting or reassociating.
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// Fast2Sum: exact when the exponent of a is not below that of b.
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

struct PolDF64 {
  using Elem = float4;   // (re.hi, re.lo, im.hi, im.lo)
  using Real = DF;
  using Coef = float2;   // (hi, lo) split of an FP64 coefficient, made on the host
  static constexpr int kSwizzle = 7;
  static constexpr int kSwShift = 0;
  static __device__ __forceinline__ Coef coef(const double* c, int i) {
    return reinterpret_cast<const float2*>(c)[i];
  }
  static __device__ __forceinline__ Elem conj_if(Elem e, unsigned t) {
    e.z = __int_as_float(__float_as_int(e.z) ^ int(t << 31));
    e.w = __int_as_float(__float_as_int(e.w) ^ int(t << 31));
    return e;
  }
  static __device__ __forceinline__ Real re(const Elem& e) { return {e.x, e.y}; }
  static __device__ __forceinline__ Real im(const Elem& e) { return {e.z, e.w}; }
  static __device__ __forceinline__ Elem make(Real r, Real i) { return make_float4(r.hi, r.lo, i.hi, i.lo); }
  static __device__ __forceinline__ Elem conj(Elem e) { e.z = -e.z; e.w = -e.w; return e; }
  static __device__ __forceinline__ Real add(Real a, Real b) {
    DF s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
  }
  static __device__ __forceinline__ Real neg(Real a) { return {-a.hi, -a.lo}; }
  static __device__ __forceinline__ Real flip(Real a) {
    return {__int_as_float(__float_as_int(a.hi) ^ int(0x80000000u)),
            __int_as_float(__float_as_int(a.lo) ^ int(0x80000000u))};
  }
  static __device__ __forceinline__ Real sub(Real a, Real b) { return add(a, neg(b)); }
  static __device__ __forceinline__ Real half(Real a) { return {__fmul_rn(0.5f, a.hi), __fmul_rn(0.5f, a.lo)}; }
  // x * c with the exact rounding error of the leading product (TwoProduct by FMA)
  // and the two cross terms; the lo * lo term is below the format's precision.
  static __device__ __forceinline__ Real mul(Real x, Coef c) {
    float p = __fmul_rn(x.hi, c.x);
    float e = __fmaf_rn(x.hi, c.x, -p);
    e = __fmaf_rn(x.hi, c.y, e);
    e = __fmaf_rn(x.lo, c.x, e);
    return {p, e};   // unnormalised; norm() or add() renormalises
  }
  // acc + x * c, left unnormalised (|lo| may exceed half an ulp of hi); the
  // leading-part sum is exact (TwoSum), so nothing is lost by deferring.
  static __device__ __forceinline__ Real mac(Real acc, Real x, Coef c) {
    float p = __fmul_rn(x.hi, c.x);
    float e = __fmaf_rn(x.hi, c.x, -p);
    e = __fmaf_rn(x.hi, c.y, e);
    e = __fmaf_rn(x.lo, c.x, e);
    DF s = df_two_sum(acc.hi, p);
    return {s.hi, __fadd_rn(s.lo, __fadd_rn(e, acc.lo))};
  }
  static __device__ __forceinline__ Real norm(Real a) { return df_fast_two_sum(a.hi, a.lo); }
  static __device__ __forceinline__ double to_double(Real a) { return (double)a.hi + (double)a.lo; }
};

template <class P>
struct Cx {
  typename P::Real re, im;
};

}  // namespace orkan
