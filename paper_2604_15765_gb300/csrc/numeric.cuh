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
//
// A PolDF64 element is stored as (re.hi, im.hi, re.lo, im.lo): one 16-byte
// load yields the pairs (re.hi, im.hi) and (re.lo, im.lo), which the hot op
// bodies feed to Blackwell's paired FP32 instructions (f32x2: one instruction
// per two lanes), so that the real and imaginary parts of a complex value
// share every double-float step.
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
  using Elem = float4;   // (re.hi, im.hi, re.lo, im.lo)
  using Real = DF;
  using Coef = float2;   // (hi, lo) split of an FP64 coefficient, made on the host
  static constexpr int kSwizzle = 7;
  static constexpr int kSwShift = 0;
  static __device__ __forceinline__ Coef coef(const double* c, int i) {
    return reinterpret_cast<const float2*>(c)[i];
  }
  static __device__ __forceinline__ Elem conj_if(Elem e, unsigned t) {
    e.y = __int_as_float(__float_as_int(e.y) ^ int(t << 31));
    e.w = __int_as_float(__float_as_int(e.w) ^ int(t << 31));
    return e;
  }
  static __device__ __forceinline__ Real re(const Elem& e) { return {e.x, e.z}; }
  static __device__ __forceinline__ Real im(const Elem& e) { return {e.y, e.w}; }
  static __device__ __forceinline__ Elem make(Real r, Real i) { return make_float4(r.hi, i.hi, r.lo, i.lo); }
  static __device__ __forceinline__ Elem conj(Elem e) { e.y = -e.y; e.w = -e.w; return e; }
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

// ------------------------------------------------------------------ paired double-float
// A complex double-float value with its real and imaginary parts in the two
// lanes of f32x2 operands: hi = (re.hi, im.hi), lo = (re.lo, im.lo).  Every
// operation is the PolDF64 operation above applied to both lanes at once
// (same rounding, same results), with half the instructions.
struct DF2 {
  float2 hi, lo;
};

__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __fadd2_rn(a, f2neg(b)); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2swap(float2 a) { return make_float2(a.y, a.x); }

// Fast2Sum on both lanes (exact when |a| >= |b| lane-wise or a == 0).
__device__ __forceinline__ DF2 df2_fast(float2 a, float2 b) {
  const float2 s = f2add(a, b);
  return {s, f2sub(b, f2sub(s, a))};
}
// a + b.  The leading parts are summed by TwoSum, the trailing parts with
// the error, then renormalised (11 paired instructions).
__device__ __forceinline__ DF2 df2_add(const DF2& a, const DF2& b) {
  const float2 s = f2add(a.hi, b.hi);
  const float2 bb = f2sub(s, a.hi);
  const float2 e = f2add(f2sub(a.hi, f2sub(s, bb)), f2sub(b.hi, bb));
  return df2_fast(s, f2add(e, f2add(a.lo, b.lo)));
}
__device__ __forceinline__ DF2 df2_neg(const DF2& a) { return {f2neg(a.hi), f2neg(a.lo)}; }
__device__ __forceinline__ DF2 df2_sub(const DF2& a, const DF2& b) { return df2_add(a, df2_neg(b)); }
// a + s * b with a lane-wise sign pair s = (+-1, +-1): the product by +-1 is
// exact, so each FMA below rounds like the add it replaces (same cost as df2_add).
__device__ __forceinline__ DF2 df2_add_signed(const DF2& a, const DF2& b, float2 sg) {
  const float2 s = f2fma(b.hi, sg, a.hi);
  const float2 bb = f2sub(s, a.hi);
  const float2 e = f2add(f2sub(a.hi, f2sub(s, bb)), f2fma(b.hi, sg, f2neg(bb)));
  return df2_fast(s, f2add(e, f2fma(b.lo, sg, a.lo)));
}
// a + i b and a - i b: i b = (-b.im, b.re), the lane swap of b with sign (-1, +1).
__device__ __forceinline__ DF2 df2_add_i(const DF2& a, const DF2& b) {
  return df2_add_signed(a, DF2{f2swap(b.hi), f2swap(b.lo)}, make_float2(-1.0f, 1.0f));
}
__device__ __forceinline__ DF2 df2_sub_i(const DF2& a, const DF2& b) {
  return df2_add_signed(a, DF2{f2swap(b.hi), f2swap(b.lo)}, make_float2(1.0f, -1.0f));
}
// x * c with TwoProduct on the leading parts and the two cross terms, left
// unnormalised; c is a coefficient pair (one factor per lane).
__device__ __forceinline__ DF2 df2_mul(const DF2& x, const DF2& c) {
  const float2 p = f2mul(x.hi, c.hi);
  float2 e = f2fma(x.hi, c.hi, f2neg(p));
  e = f2fma(x.hi, c.lo, e);
  e = f2fma(x.lo, c.hi, e);
  return {p, e};
}
// acc + x * c, unnormalised like PolDF64::mac (12 paired instructions).
__device__ __forceinline__ DF2 df2_mac(const DF2& acc, const DF2& x, const DF2& c) {
  const float2 p = f2mul(x.hi, c.hi);
  float2 e = f2fma(x.hi, c.hi, f2neg(p));
  e = f2fma(x.hi, c.lo, e);
  e = f2fma(x.lo, c.hi, e);
  const float2 s = f2add(acc.hi, p);
  const float2 bb = f2sub(s, acc.hi);
  const float2 ee = f2add(f2sub(acc.hi, f2sub(s, bb)), f2sub(p, bb));
  return {s, f2add(ee, f2add(e, acc.lo))};
}
// acc + (lane swap of x) * c: with c = (-v, v) this adds v * (i x), with
// c = (v, -v) it adds -v * (i x).
__device__ __forceinline__ DF2 df2_mac_swap(const DF2& acc, const DF2& x, const DF2& c) {
  return df2_mac(acc, DF2{f2swap(x.hi), f2swap(x.lo)}, c);
}
__device__ __forceinline__ DF2 df2_norm(const DF2& a) { return df2_fast(a.hi, a.lo); }
__device__ __forceinline__ DF2 df2_half(const DF2& a) {
  const float2 h = make_float2(0.5f, 0.5f);
  return {f2mul(a.hi, h), f2mul(a.lo, h)};
}

// Conversions between the per-part form Cx<PolDF64> and the paired form.
__device__ __forceinline__ DF2 to_df2(const Cx<PolDF64>& z) {
  return {make_float2(z.re.hi, z.im.hi), make_float2(z.re.lo, z.im.lo)};
}
__device__ __forceinline__ Cx<PolDF64> from_df2(const DF2& z) {
  return Cx<PolDF64>{DF{z.hi.x, z.lo.x}, DF{z.hi.y, z.lo.y}};
}
// Coefficient pair k of a paired coefficient list: two 8-byte slots,
// (c0.hi, c1.hi) then (c0.lo, c1.lo), written by the host.
__device__ __forceinline__ DF2 pcoef(const double* cf, int k) {
  const float2* p = reinterpret_cast<const float2*>(cf);
  return {p[2 * k], p[2 * k + 1]};
}

}  // namespace orkan
