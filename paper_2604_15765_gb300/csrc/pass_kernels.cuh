// Fused k-local conjugation passes over the tiled lower-triangle layout.
//
// Sec. III-B stores tiles T[ti, tj], ti >= tj, row-major, elements row-major.
// Sec. III-C splits an update into intra-tile work (all targets below m,
// Algorithm 2) and cross-tile work (a target a >= m couples the tiles whose
// indices differ in bit a - m, Algorithm 3, with subcases A / B / C depending
// on whether the partner tile T[ti0, tj1] is stored, is the adjoint of a
// stored tile, or is the adjoint of T[ti1, tj0] itself).
//
// GPU design: one CTA owns one *tile group* at a time: the 2^h x 2^h tiles
// (h = number of high qubits in the pass, 0..2) whose grid indices share the
// bits outside the high positions.  The group is staged in shared memory in
// its *logical* orientation: a tile of the group that lies in the upper
// triangle is loaded from its stored partner transposed and conjugated
// (this covers subcases B and C uniformly), so that every op of the fused
// pass sees a plain (2^h M) x (2^h M) hermitian block and applies Eq. (2) to
// its 2^k x 2^k sub-blocks.  Only stored tiles are written back, each exactly
// once: in a diagonal group (ti == tj before bit insertion) the upper slots
// are mirrors of lower slots of the same group and are not written.
//
// Shared memory holds each slot row-major with the 16-byte (8-byte) element
// index XOR-swizzled by the row, so that transposed loads/stores and
// strided butterfly accesses hit distinct banks.
#pragma once
#include "orkan_internal.h"
#include "numeric.cuh"
#include "device_util.cuh"
#include <type_traits>

namespace orkan {
namespace {

// Subroutine 1 with a zero bit: make room at position p.
__device__ __forceinline__ int64_t ins0(int64_t x, int p) {
  const int64_t low = x & ((int64_t(1) << p) - 1);
  return ((x >> p) << (p + 1)) | low;
}
__device__ __forceinline__ int ins0i(int x, int p) {
  const int low = x & ((1 << p) - 1);
  return ((x >> p) << (p + 1)) | low;
}

// Group layout in shared memory.  Logical element (li, lj) of the
// (2^H R) x (2^H M) group, li = x R + r, lj = y M + c, lives in slot (x, y)
// at row r; the element (16-byte granule) index inside a row is
// XOR-swizzled with the row so that row-wise and column-wise walks hit
// distinct banks:
//   idx = ((x 2^H + y) R + r) M + (c ^ swz(r)),
//   swz(r) = ((r & sw) ^ (bit 3 of r ? b3 : 0)) << SH.
// With 16-byte elements in slots of at least 16 rows, b3 = 7: rows with bit 3
// set flip all three low granule bits.  Then any eight rows with one of the
// bits 0..2 clear (the first rows of the 2x2 blocks of a single-qubit op on
// that bit, walked rows-first) still cover all eight 16-byte bank groups,
// which the plain row XOR cannot: it keeps that bit clear.  swz is linear
// over GF(2), so a row partner's swizzle is swz(r) ^ swz(2^pos).
// Slots whose tile lies in the upper triangle are loaded already transposed
// and conjugated, so every op sees plain logical elements.
template <class P, int H, int MLOG, int RL>
struct GMap {
  static constexpr int M = 1 << MLOG;
  static constexpr int R = 1 << RL;
  static constexpr int SH = P::kSwShift;
  static constexpr int SW = ((M >> SH) - 1) < 7 ? ((M >> SH) - 1) : 7;
  static constexpr int B3 = (SH == 0 && R >= 16) ? SW : 0;
  static __host__ __device__ __forceinline__ constexpr int swz(int r) {
    return ((r & SW) ^ (((r >> 3) & 1) ? B3 : 0)) << SH;
  }
  static __device__ __forceinline__ int idx(int li, int lj) {
    const int x = li >> RL, r = li & (R - 1);
    const int y = lj >> MLOG, c = lj & (M - 1);
    return ((((x << H) | y) << RL | r) << MLOG) + (c ^ swz(r));
  }
  // index of the partner whose row (or column) index has bit `pos` set, as
  // idx' = (idx + add) ^ xr, for an element whose index has that bit clear
  static __device__ __forceinline__ void row_delta(int pos, int& add, int& xr) {
    if (pos < RL) { add = (1 << pos) << MLOG; xr = swz(1 << pos); }
    else { add = (1 << (pos - RL)) << (H + RL + MLOG); xr = 0; }
  }
  static __device__ __forceinline__ void col_delta(int pos, int& add, int& xr) {
    if (pos < MLOG) { add = 0; xr = 1 << pos; }
    else { add = (1 << (pos - MLOG)) << (RL + MLOG); xr = 0; }
  }
};

template <class P>
__device__ __forceinline__ Cx<P> ld(const typename P::Elem* sm, int i) {
  const auto e = sm[i];
  return Cx<P>{P::re(e), P::im(e)};
}
template <class P>
__device__ __forceinline__ void st(typename P::Elem* sm, int i, const Cx<P>& v) {
  sm[i] = P::make(v.re, v.im);
}

// ------------------------------------------------------------------ op bodies
// A 2x2 block [[a, b], [c, d]] in Pauli coordinates s_k = 2 z_k:
//   s0 = a + d, s1 = b + c, s2 = i (b - c), s3 = a - d,
// and back: a = z0 + z3, d = z0 - z3, b = z1 - i z2, c = z1 + i z2.

template <class P>
__device__ __forceinline__ void body_ptm1(Cx<P>& a, Cx<P>& b, Cx<P>& c, Cx<P>& d, const double* cf) {
  using R = typename P::Real;
  R sr[4], si[4];
  sr[0] = P::add(a.re, d.re); si[0] = P::add(a.im, d.im);
  sr[1] = P::add(b.re, c.re); si[1] = P::add(b.im, c.im);
  sr[2] = P::sub(c.im, b.im); si[2] = P::sub(b.re, c.re);
  sr[3] = P::sub(a.re, d.re); si[3] = P::sub(a.im, d.im);
  R zr[4], zi[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    R ar = P::mul(sr[0], P::coef(cf, 4 * i));
    R ai = P::mul(si[0], P::coef(cf, 4 * i));
#pragma unroll
    for (int j = 1; j < 4; ++j) {
      ar = P::mac(ar, sr[j], P::coef(cf, 4 * i + j));
      ai = P::mac(ai, si[j], P::coef(cf, 4 * i + j));
    }
    zr[i] = P::norm(ar);
    zi[i] = P::norm(ai);
  }
  a.re = P::add(zr[0], zr[3]); a.im = P::add(zi[0], zi[3]);
  d.re = P::sub(zr[0], zr[3]); d.im = P::sub(zi[0], zi[3]);
  b.re = P::add(zr[1], zi[2]); b.im = P::sub(zi[1], zr[2]);
  c.re = P::sub(zr[1], zi[2]); c.im = P::add(zi[1], zr[2]);
}

template <class P>
__device__ __forceinline__ void body_ptm1_u(Cx<P>& a, Cx<P>& b, Cx<P>& c, Cx<P>& d, const double* cf) {
  using R = typename P::Real;
  R sr[3], si[3];
  sr[0] = P::add(b.re, c.re); si[0] = P::add(b.im, c.im);
  sr[1] = P::sub(c.im, b.im); si[1] = P::sub(b.re, c.re);
  sr[2] = P::sub(a.re, d.re); si[2] = P::sub(a.im, d.im);
  const R z0r = P::half(P::add(a.re, d.re)), z0i = P::half(P::add(a.im, d.im));
  R zr[3], zi[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R ar = P::mul(sr[0], P::coef(cf, 3 * i));
    R ai = P::mul(si[0], P::coef(cf, 3 * i));
#pragma unroll
    for (int j = 1; j < 3; ++j) {
      ar = P::mac(ar, sr[j], P::coef(cf, 3 * i + j));
      ai = P::mac(ai, si[j], P::coef(cf, 3 * i + j));
    }
    zr[i] = P::norm(ar);
    zi[i] = P::norm(ai);
  }
  a.re = P::add(z0r, zr[2]); a.im = P::add(z0i, zi[2]);
  d.re = P::sub(z0r, zr[2]); d.im = P::sub(z0i, zi[2]);
  b.re = P::add(zr[0], zi[1]); b.im = P::sub(zi[0], zr[1]);
  c.re = P::sub(zr[0], zi[1]); c.im = P::add(zi[0], zr[1]);
}

template <class P>
__device__ __forceinline__ void body_ptm1_ad(Cx<P>& a, Cx<P>& b, Cx<P>& c, Cx<P>& d, const double* cf) {
  using R = typename P::Real;
  const auto al = P::coef(cf, 0), be = P::coef(cf, 1), ga = P::coef(cf, 2), de = P::coef(cf, 3);
  const auto rh = P::coef(cf, 4), sg = P::coef(cf, 5);
  const R ar = P::norm(P::mac(P::mul(a.re, al), d.re, be));
  const R ai = P::norm(P::mac(P::mul(a.im, al), d.im, be));
  const R dr = P::norm(P::mac(P::mul(a.re, ga), d.re, de));
  const R di = P::norm(P::mac(P::mul(a.im, ga), d.im, de));
  if constexpr (std::is_same<R, double>::value) {
    // native FP64 (2 operations per SM per clock on GB300): the named channels
    // and projectors scale h01 / h10 by a real factor (sig = 0, uniform over
    // the warp), which needs 12 instead of 16 FP64 operations per block
    if (sg == 0.0) {
      a.re = ar; a.im = ai; d.re = dr; d.im = di;
      b.re = P::mul(b.re, rh); b.im = P::mul(b.im, rh);
      c.re = P::mul(c.re, rh); c.im = P::mul(c.im, rh);
      return;
    }
  }
  // h01' = (rho - i sig) h01, h10' = (rho + i sig) h10
  const R br = P::norm(P::mac(P::mul(b.re, rh), b.im, sg));
  const R bi = P::norm(P::mac(P::mul(b.im, rh), P::neg(b.re), sg));
  const R cr = P::norm(P::mac(P::mul(c.re, rh), P::neg(c.im), sg));
  const R ci = P::norm(P::mac(P::mul(c.im, rh), c.re, sg));
  a.re = ar; a.im = ai; d.re = dr; d.im = di;
  b.re = br; b.im = bi; c.re = cr; c.im = ci;
}

// Integer codes of monomial ops are stored as raw 64-bit integers in their slots.
__device__ __forceinline__ int icoef(const double* cf, int i) {
  return int(reinterpret_cast<const long long*>(cf)[i]);
}

// z * i^k for k = 0..3: exact (swaps and sign-bit flips of the parts, no
// floating-point instructions).
template <class P>
__device__ __forceinline__ Cx<P> rot_i(const Cx<P>& z, int k) {
  switch (k & 3) {
    case 0: return z;
    case 1: return Cx<P>{P::flip(z.im), z.re};
    case 2: return Cx<P>{P::flip(z.re), P::flip(z.im)};
    default: return Cx<P>{z.im, P::flip(z.re)};
  }
}

// Monomial single-qubit unitary V[i][p_i] = i^{q_i}: (V h V^dagger)[i][j] =
// i^{q_i - q_j} h[p_i][p_j].
template <class P>
__device__ __forceinline__ void body_mono1(Cx<P>& a, Cx<P>& b, Cx<P>& c, Cx<P>& d, const double* cf) {
  const int p0 = icoef(cf, 0), p1 = icoef(cf, 1), q0 = icoef(cf, 2), q1 = icoef(cf, 3);
  const Cx<P> h00 = a, h01 = b, h10 = c, h11 = d;
  auto pick = [&](int r, int s) -> Cx<P> {
    return r ? (s ? h11 : h10) : (s ? h01 : h00);
  };
  a = rot_i<P>(pick(p0, p0), q0 - q0);
  b = rot_i<P>(pick(p0, p1), q0 - q1);
  c = rot_i<P>(pick(p1, p0), q1 - q0);
  d = rot_i<P>(pick(p1, p1), q1 - q1);
}

// Forward / inverse single-qubit Pauli transform on four complex values.
template <class P>
__device__ __forceinline__ void pauli_fwd(Cx<P>& a, Cx<P>& b, Cx<P>& c, Cx<P>& d) {
  Cx<P> s0{P::add(a.re, d.re), P::add(a.im, d.im)};
  Cx<P> s1{P::add(b.re, c.re), P::add(b.im, c.im)};
  Cx<P> s2{P::sub(c.im, b.im), P::sub(b.re, c.re)};
  Cx<P> s3{P::sub(a.re, d.re), P::sub(a.im, d.im)};
  a = s0; b = s1; c = s2; d = s3;
}
template <class P>
__device__ __forceinline__ void pauli_inv(Cx<P>& z0, Cx<P>& z1, Cx<P>& z2, Cx<P>& z3) {
  Cx<P> a{P::add(z0.re, z3.re), P::add(z0.im, z3.im)};
  Cx<P> d{P::sub(z0.re, z3.re), P::sub(z0.im, z3.im)};
  Cx<P> b{P::add(z1.re, z2.im), P::sub(z1.im, z2.re)};
  Cx<P> c{P::sub(z1.re, z2.im), P::add(z1.im, z2.re)};
  z0 = a; z1 = b; z2 = c; z3 = d;
}


// Generic two-qubit map in the two-qubit Pauli basis (coefficients R / 4),
// all in registers.  Element (ra, ca) of the block, ra = r0 + 2 r1, sits in
// h[4 ra + ca]; the forward transform runs over bit 0 (r0, c0), then bit 1.
template <class P>
__device__ __forceinline__ void body_ptm2(Cx<P> (&h)[16], const double* cf) {
  using R = typename P::Real;
#pragma unroll
  for (int r1 = 0; r1 < 2; ++r1)
#pragma unroll
    for (int c1 = 0; c1 < 2; ++c1)
      pauli_fwd<P>(h[(2 * r1) * 4 + 2 * c1], h[(2 * r1) * 4 + 2 * c1 + 1], h[(2 * r1 + 1) * 4 + 2 * c1],
                   h[(2 * r1 + 1) * 4 + 2 * c1 + 1]);
#pragma unroll
  for (int a0 = 0; a0 < 4; ++a0) {
    const int o = (a0 >> 1) * 4 + (a0 & 1);
    pauli_fwd<P>(h[o], h[o + 2], h[o + 8], h[o + 10]);
  }
  // h[sidx(a)] now holds s_a, a = a0 + 4 a1
  constexpr int sidx[16] = {0, 1, 4, 5, 2, 3, 6, 7, 8, 9, 12, 13, 10, 11, 14, 15};
  Cx<P> z[16];
#pragma unroll
  for (int a = 0; a < 16; ++a) {
    R zr = P::mul(h[sidx[0]].re, P::coef(cf, 16 * a));
    R zi = P::mul(h[sidx[0]].im, P::coef(cf, 16 * a));
#pragma unroll
    for (int b = 1; b < 16; ++b) {
      zr = P::mac(zr, h[sidx[b]].re, P::coef(cf, 16 * a + b));
      zi = P::mac(zi, h[sidx[b]].im, P::coef(cf, 16 * a + b));
    }
    z[a] = Cx<P>{P::norm(zr), P::norm(zi)};
  }
#pragma unroll
  for (int a = 0; a < 16; ++a) h[sidx[a]] = z[a];
#pragma unroll
  for (int a0 = 0; a0 < 4; ++a0) {
    const int o = (a0 >> 1) * 4 + (a0 & 1);
    pauli_inv<P>(h[o], h[o + 2], h[o + 8], h[o + 10]);
  }
#pragma unroll
  for (int r1 = 0; r1 < 2; ++r1)
#pragma unroll
    for (int c1 = 0; c1 < 2; ++c1)
      pauli_inv<P>(h[(2 * r1) * 4 + 2 * c1], h[(2 * r1) * 4 + 2 * c1 + 1], h[(2 * r1 + 1) * 4 + 2 * c1],
                   h[(2 * r1 + 1) * 4 + 2 * c1 + 1]);
}

// out[i] = sum_k A[i][k] in[k] for the 4x4 complex A = V (CONJ = false) or
// conj(V) (CONJ = true); V row-major, re/im interleaved in the coefficients.
template <class P, bool CONJ>
__device__ __forceinline__ void matvec4(const Cx<P> (&in)[4], Cx<P> (&out)[4], const double* cf) {
  using R = typename P::Real;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    R accr, acci;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const auto ar = P::coef(cf, 2 * (4 * i + k)), ai = P::coef(cf, 2 * (4 * i + k) + 1);
      // V:       re += ar xr - ai xi,  im += ar xi + ai xr
      // conj(V): re += ar xr + ai xi,  im += ar xi - ai xr
      const R xr = in[k].re, xi = in[k].im;
      if (k == 0) {
        accr = P::mul(xr, ar);
        acci = P::mul(xi, ar);
      } else {
        accr = P::mac(accr, xr, ar);
        acci = P::mac(acci, xi, ar);
      }
      accr = P::mac(accr, CONJ ? xi : P::neg(xi), ai);
      acci = P::mac(acci, CONJ ? P::neg(xr) : xr, ai);
    }
    out[i] = Cx<P>{P::norm(accr), P::norm(acci)};
  }
}

// out[i] = i^{q_i} in[p_i] (V) or out[j] = i^{-q_j} in[p_j] (conj(V) applied as
// h V^dagger on a row): the monomial form of matvec4, no arithmetic.
template <class P, bool CONJ>
__device__ __forceinline__ void matvec4_mono(const Cx<P> (&in)[4], Cx<P> (&out)[4], const double* cf) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int p = icoef(cf, i), q = icoef(cf, 4 + i);
    const Cx<P> x = p == 0 ? in[0] : (p == 1 ? in[1] : (p == 2 ? in[2] : in[3]));
    out[i] = rot_i<P>(x, CONJ ? -q : q);
  }
}

// Two-qubit unitary, h <- V h V^dagger, on a 4x4 block in registers: every
// row becomes h[k, :] V^dagger, then every column V (.)[:, j] (Eq. 2 with
// one Kraus operator).  MONO: the monomial form (codes after the dense V).
template <class P, bool MONO>
__device__ __forceinline__ void body_u2(Cx<P> (&h)[16], const double* cf) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    Cx<P> in[4], out[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) in[l] = h[4 * k + l];
    if constexpr (MONO) matvec4_mono<P, true>(in, out, cf + 32);
    else matvec4<P, true>(in, out, cf);
#pragma unroll
    for (int l = 0; l < 4; ++l) h[4 * k + l] = out[l];
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    Cx<P> in[4], out[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) in[l] = h[4 * l + j];
    if constexpr (MONO) matvec4_mono<P, false>(in, out, cf + 32);
    else matvec4<P, false>(in, out, cf);
#pragma unroll
    for (int l = 0; l < 4; ++l) h[4 * l + j] = out[l];
  }
}

// ------------------------------------------------------------------ paired double-float bodies
// The PolDF64 forms of the single-qubit bodies above: the same operations in
// the same order on both parts of each complex value at once (f32x2), so the
// results equal the per-part forms bit for bit.  Their coefficient lists are
// paired (pcoef, written by the host): a real coefficient c as the pair
// (c, c); where the per-part form multiplies i t (t a complex value), the
// pair (-c, c) multiplies the lane swap (t.im, t.re) instead, which gives
// c (i t) without forming i t.
//
// The two-qubit sweeps (matvec4) stay per-part.  Paired, they issued 29 %
// fewer instructions but ran no faster: merging the real and imaginary
// chains halves the independent work per thread, the unit loop then has to
// stay rolled to avoid spills, and with four warps per scheduler the pass
// becomes latency-bound (measured on a two-high-qubit unitary pass, n = 13).

template <>
__device__ __forceinline__ void body_ptm1<PolDF64>(Cx<PolDF64>& a, Cx<PolDF64>& b, Cx<PolDF64>& c,
                                                   Cx<PolDF64>& d, const double* cf) {
  // coefficient pairs 4 i + j: R_ij / 2, the j = 2 column as (-R, R)
  const DF2 A = to_df2(a), B = to_df2(b), C = to_df2(c), D = to_df2(d);
  const DF2 s0 = df2_add(A, D), s1 = df2_add(B, C), t = df2_sub(B, C), s3 = df2_sub(A, D);
  DF2 z[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    DF2 acc = df2_mul(s0, pcoef(cf, 4 * i));
    acc = df2_mac(acc, s1, pcoef(cf, 4 * i + 1));
    acc = df2_mac_swap(acc, t, pcoef(cf, 4 * i + 2));
    acc = df2_mac(acc, s3, pcoef(cf, 4 * i + 3));
    z[i] = df2_norm(acc);
  }
  a = from_df2(df2_add(z[0], z[3]));
  d = from_df2(df2_sub(z[0], z[3]));
  b = from_df2(df2_sub_i(z[1], z[2]));
  c = from_df2(df2_add_i(z[1], z[2]));
}

template <>
__device__ __forceinline__ void body_ptm1_u<PolDF64>(Cx<PolDF64>& a, Cx<PolDF64>& b, Cx<PolDF64>& c,
                                                     Cx<PolDF64>& d, const double* cf) {
  // coefficient pairs 3 i + j: R3_ij / 2, the j = 1 column as (-R, R)
  const DF2 A = to_df2(a), B = to_df2(b), C = to_df2(c), D = to_df2(d);
  const DF2 s0 = df2_add(B, C), t = df2_sub(B, C), s2 = df2_sub(A, D);
  const DF2 z0 = df2_half(df2_add(A, D));
  DF2 z[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    DF2 acc = df2_mul(s0, pcoef(cf, 3 * i));
    acc = df2_mac_swap(acc, t, pcoef(cf, 3 * i + 1));
    acc = df2_mac(acc, s2, pcoef(cf, 3 * i + 2));
    z[i] = df2_norm(acc);
  }
  a = from_df2(df2_add(z0, z[2]));
  d = from_df2(df2_sub(z0, z[2]));
  b = from_df2(df2_sub_i(z[0], z[1]));
  c = from_df2(df2_add_i(z[0], z[1]));
}

template <>
__device__ __forceinline__ void body_ptm1_ad<PolDF64>(Cx<PolDF64>& a, Cx<PolDF64>& b, Cx<PolDF64>& c,
                                                      Cx<PolDF64>& d, const double* cf) {
  // pairs: al, be, ga, de, rho as (c, c); then (-sig, sig) and (sig, -sig)
  const DF2 A = to_df2(a), B = to_df2(b), C = to_df2(c), D = to_df2(d);
  const DF2 rh = pcoef(cf, 4);
  a = from_df2(df2_norm(df2_mac(df2_mul(A, pcoef(cf, 0)), D, pcoef(cf, 1))));
  d = from_df2(df2_norm(df2_mac(df2_mul(A, pcoef(cf, 2)), D, pcoef(cf, 3))));
  // h01' = (rho - i sig) h01, h10' = (rho + i sig) h10
  b = from_df2(df2_norm(df2_mac_swap(df2_mul(B, rh), B, pcoef(cf, 6))));
  c = from_df2(df2_norm(df2_mac_swap(df2_mul(C, rh), C, pcoef(cf, 5))));
}

// ------------------------------------------------------------------ op drivers
// Every driver walks its units with a compile-time count per thread (the
// unit count is a power of two fixed by the geometry), and is instantiated
// per op form, so the element loops carry no bounds or form branches.
// ROLLED keeps the unit loop rolled (the kernels that also hold the large
// generic two-qubit body, where unrolling would spill).
template <int ITERS, bool ROLLED, class F>
__device__ __forceinline__ void for_units(F&& unit) {
  if constexpr (ROLLED) {
#pragma unroll 1
    for (int k = 0; k < ITERS; ++k) unit(k);
  } else {
#pragma unroll
    for (int k = 0; k < ITERS; ++k) unit(k);
  }
}

template <class P, class G, int NT, int rows_log2g, int cols_log2g, bool ROLLED, int FORM>
__device__ __forceinline__ void apply_1q_form(typename P::Elem* sm, const G& gm, const PassOp& op,
                                              const double* cf) {
  constexpr int ncb_log2 = cols_log2g - 1, nrb_log2 = rows_log2g - 1;
  constexpr int nb = 1 << (nrb_log2 + ncb_log2);
  constexpr int iters = (nb + NT - 1) / NT;
  // where the bit-3 swizzle is on (16-byte elements, slots of >= 16 rows),
  // consecutive threads take consecutive block rows of one block column,
  // which is then conflict-free for every target bit; otherwise consecutive
  // block columns of one block row
  constexpr bool rows_first = G::B3 != 0;
  int ra, rx, ca, cx;
  gm.row_delta(op.rbit[0], ra, rx);
  gm.col_delta(op.cbit[0], ca, cx);
  for_units<iters, ROLLED>([&](int k) {
    const int b = int(threadIdx.x) + k * NT;
    if (nb % NT == 0 || b < nb) {
      const int cb = rows_first ? b >> nrb_log2 : b & ((1 << ncb_log2) - 1);
      const int rb = rows_first ? b & ((1 << nrb_log2) - 1) : b >> ncb_log2;
      const int c0 = ins0i(cb, op.cbit[0]);
      const int r0 = ins0i(rb, op.rbit[0]);
      const int i00 = gm.idx(r0, c0);
      const int i01 = (i00 + ca) ^ cx, i10 = (i00 + ra) ^ rx;
      const int i11 = (i10 + ca) ^ cx;
      Cx<P> a = ld<P>(sm, i00), bb = ld<P>(sm, i01), c = ld<P>(sm, i10), d = ld<P>(sm, i11);
      if constexpr (FORM == OP_PTM1_U) body_ptm1_u<P>(a, bb, c, d, cf);
      else if constexpr (FORM == OP_PTM1_AD) body_ptm1_ad<P>(a, bb, c, d, cf);
      else if constexpr (FORM == OP_MONO1) body_mono1<P>(a, bb, c, d, cf);
      else body_ptm1<P>(a, bb, c, d, cf);
      st<P>(sm, i00, a);
      st<P>(sm, i01, bb);
      st<P>(sm, i10, c);
      st<P>(sm, i11, d);
    }
  });
}

template <class P, class G, int NT, int rows_log2g, int cols_log2g, bool ROLLED = false>
__device__ __forceinline__ void apply_1q(typename P::Elem* sm, const G& gm, const PassOp& op, const double* coef) {
  const double* cf = coef + op.coef;
  switch (op.kind) {
    case OP_PTM1_U: apply_1q_form<P, G, NT, rows_log2g, cols_log2g, ROLLED, OP_PTM1_U>(sm, gm, op, cf); break;
    case OP_PTM1_AD: apply_1q_form<P, G, NT, rows_log2g, cols_log2g, ROLLED, OP_PTM1_AD>(sm, gm, op, cf); break;
    case OP_MONO1: apply_1q_form<P, G, NT, rows_log2g, cols_log2g, ROLLED, OP_MONO1>(sm, gm, op, cf); break;
    default: apply_1q_form<P, G, NT, rows_log2g, cols_log2g, ROLLED, OP_PTM1>(sm, gm, op, cf); break;
  }
}

// Two-qubit unitary as two separable sweeps (V h V^dagger = V (h V^dagger)):
// every row gets h[r, :] <- h[r, :] V^dagger on the column bits, then every
// column gets h[:, c] <- V h[:, c] on the row bits.  Same 32 multiply-adds per
// element as the block form, in 4-element units (small code, few registers).
template <class P, class G, int NT, int rows_log2g, int cols_log2g, bool ROLLED, bool MONO>
__device__ __forceinline__ void apply_u2_sep_form(typename P::Elem* sm, const G& gm, const PassOp& op,
                                                  const double* cf) {
  {
    int a0, x0, a1, x1;
    gm.col_delta(op.cbit[0], a0, x0);
    gm.col_delta(op.cbit[1], a1, x1);
    constexpr int nc_log2 = cols_log2g - 2;
    constexpr int nu = 1 << (rows_log2g + nc_log2);
    constexpr int iters = (nu + NT - 1) / NT;
    for_units<iters, ROLLED>([&](int k) {
      const int u = int(threadIdx.x) + k * NT;
      if (nu % NT == 0 || u < nu) {
        const int li = u >> nc_log2;
        const int c0 = ins0i(ins0i(u & ((1 << nc_log2) - 1), op.cbit[0]), op.cbit[1]);
        int ix[4];
        ix[0] = gm.idx(li, c0);
        ix[1] = (ix[0] + a0) ^ x0;
        ix[2] = (ix[0] + a1) ^ x1;
        ix[3] = (ix[1] + a1) ^ x1;
        Cx<P> in[4], out[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) in[a] = ld<P>(sm, ix[a]);
        if constexpr (MONO) matvec4_mono<P, true>(in, out, cf + 32);
        else matvec4<P, true>(in, out, cf);
#pragma unroll
        for (int a = 0; a < 4; ++a) st<P>(sm, ix[a], out[a]);
      }
    });
  }
  __syncthreads();
  {
    int a0, x0, a1, x1;
    gm.row_delta(op.rbit[0], a0, x0);
    gm.row_delta(op.rbit[1], a1, x1);
    constexpr int nu = 1 << (rows_log2g - 2 + cols_log2g);
    constexpr int iters = (nu + NT - 1) / NT;
    for_units<iters, ROLLED>([&](int k) {
      const int u = int(threadIdx.x) + k * NT;
      if (nu % NT == 0 || u < nu) {
        const int lj = u & ((1 << cols_log2g) - 1);
        const int r0 = ins0i(ins0i(u >> cols_log2g, op.rbit[0]), op.rbit[1]);
        int ix[4];
        ix[0] = gm.idx(r0, lj);
        ix[1] = (ix[0] + a0) ^ x0;
        ix[2] = (ix[0] + a1) ^ x1;
        ix[3] = (ix[1] + a1) ^ x1;
        Cx<P> in[4], out[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) in[a] = ld<P>(sm, ix[a]);
        if constexpr (MONO) matvec4_mono<P, false>(in, out, cf + 32);
        else matvec4<P, false>(in, out, cf);
#pragma unroll
        for (int a = 0; a < 4; ++a) st<P>(sm, ix[a], out[a]);
      }
    });
  }
}

template <class P, class G, int NT, int rows_log2g, int cols_log2g, bool ROLLED = false>
__device__ __forceinline__ void apply_u2_sep(typename P::Elem* sm, const G& gm, const PassOp& op,
                                             const double* coef) {
  const double* cf = coef + op.coef;
  if (op.kind == OP_MONO2) apply_u2_sep_form<P, G, NT, rows_log2g, cols_log2g, ROLLED, true>(sm, gm, op, cf);
  else apply_u2_sep_form<P, G, NT, rows_log2g, cols_log2g, ROLLED, false>(sm, gm, op, cf);
}

template <class P, class G, int NT, int rows_log2g, int cols_log2g>
__device__ __forceinline__ void apply_ptm2(typename P::Elem* sm, const G& gm, const PassOp& op, const double* coef) {
  constexpr int ncb_log2 = cols_log2g - 2;
  constexpr int nb = 1 << (rows_log2g - 2 + ncb_log2);
  constexpr int iters = (nb + NT - 1) / NT;
  const double* cf = coef + op.coef;
  int ra0, rx0, ra1, rx1, ca0, cx0, ca1, cx1;
  gm.row_delta(op.rbit[0], ra0, rx0);
  gm.row_delta(op.rbit[1], ra1, rx1);
  gm.col_delta(op.cbit[0], ca0, cx0);
  gm.col_delta(op.cbit[1], ca1, cx1);
#pragma unroll 1
  for (int k = 0; k < iters; ++k) {
    const int b = int(threadIdx.x) + k * NT;
    if (nb % NT != 0 && b >= nb) break;
    const int c0 = ins0i(ins0i(b & ((1 << ncb_log2) - 1), op.cbit[0]), op.cbit[1]);
    const int r0 = ins0i(ins0i(b >> ncb_log2, op.rbit[0]), op.rbit[1]);
    int rowi[4], ix[16];
    rowi[0] = gm.idx(r0, c0);
    rowi[1] = (rowi[0] + ra0) ^ rx0;
    rowi[2] = (rowi[0] + ra1) ^ rx1;
    rowi[3] = (rowi[1] + ra1) ^ rx1;
    Cx<P> h[16];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      ix[4 * r] = rowi[r];
      ix[4 * r + 1] = (rowi[r] + ca0) ^ cx0;
      ix[4 * r + 2] = (rowi[r] + ca1) ^ cx1;
      ix[4 * r + 3] = (ix[4 * r + 1] + ca1) ^ cx1;
#pragma unroll
      for (int c = 0; c < 4; ++c) h[4 * r + c] = ld<P>(sm, ix[4 * r + c]);
    }
    body_ptm2<P>(h, cf);
#pragma unroll
    for (int t = 0; t < 16; ++t) st<P>(sm, ix[t], h[t]);
  }
}

// Rows of each tile held per work item: the largest 2^RL <= M with
// 4^H tiles x 2^RL rows x M elements within 64 KiB of shared memory per stage
// (the host planner makes the same choice; the launcher checks it).
__host__ __device__ constexpr int rows_log2_ct(int H, int MLOG, int eb) {
  int rl = 0;
  while (rl < MLOG && ((long long)(1 << (2 * H)) * (1 << MLOG) * eb << (rl + 1)) <= 64 * 1024) ++rl;
  return rl;
}

// ------------------------------------------------------------------ async copies (Ampere-style LDGSTS)
__device__ __forceinline__ void cp_async16(void* smem_ptr, const void* gmem_ptr) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_ptr));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_ptr) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem_ptr, const void* gmem_ptr) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_ptr));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_ptr) : "memory");
}
template <class E>
__device__ __forceinline__ void cp_async_elem(E* smem_ptr, const E* gmem_ptr) {
  if constexpr (sizeof(E) == 16) cp_async16(smem_ptr, gmem_ptr);
  else cp_async8(smem_ptr, gmem_ptr);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ------------------------------------------------------------------ the pass kernel
// Persistent CTAs walk the work items with a three-buffer shared-memory
// pipeline: the 16-byte asynchronous copies of items i + 1 and i + 2 are in
// flight while item i is transformed and written back, so HBM reads overlap
// the arithmetic and two items' worth of reads cover the memory latency.
constexpr int kMainThreads = 512;

// PACK: an in-tile pass (no high qubit) runs on the H = 1 geometry with four
// consecutive stored tiles as the four independent slots of a work item.
// P2: the pass contains a generic two-qubit map (PTM2); its large body is
// compiled only into these instantiations.
template <class P, int H, int MLOG, bool PACK, bool P2>
__global__ void __launch_bounds__(kMainThreads, 1)
pass_kernel(typename P::Elem* __restrict__ st, const __grid_constant__ PassDesc d) {
  using E = typename P::Elem;
  constexpr int S = 1 << H;
  constexpr int NSLOT = S * S;
  constexpr int GPE = 16 / int(sizeof(E));   // elements per 16-byte granule
  constexpr int GSH = GPE == 2 ? 1 : 0;
  constexpr int RL = rows_log2_ct(H, MLOG, int(sizeof(E)));
  using G = GMap<P, H, MLOG, RL>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // per-item slot info, four items deep: item i computes, items i+1 and i+2
  // load, item i+3 is decoded
  __shared__ int64_t s_base[4][NSLOT];
  __shared__ unsigned s_tmask[4], s_vmask[4];
  __shared__ int s_diag[4];
  E* bufs = reinterpret_cast<E*>(smem_raw);
  constexpr int m = MLOG, M = 1 << MLOG;
  constexpr int rl = RL, R = 1 << RL;
  constexpr int slot_log2 = rl + m;
  constexpr int buf_elems = NSLOT << slot_log2;
  constexpr int rows_log2g = H + rl, cols_log2g = H + m;
  const int64_t chunk_mask = (int64_t(1) << d.chunks_log2) - 1;
  const int64_t tile_elems = int64_t(1) << (2 * m);
  const G gm{};

  // slot bases, transposed / valid masks and the diagonal flag of item w (warp 0)
  auto item_info = [&](int64_t w, int b) {
    if (threadIdx.x < 32) {
      bool t = false, v = false;
      int64_t tic = 0, tjc = 0;
      if constexpr (PACK) {
        const int64_t tile = w * NSLOT + threadIdx.x;
        v = int(threadIdx.x) < NSLOT && tile < d.n_tiles;
        if (v) s_base[b][threadIdx.x] = tile * tile_elems;
      } else {
        const int64_t g = w >> d.chunks_log2;
        tic = d.skip_diag ? tri_row(g) + 1 : tri_row(g);
        tjc = d.skip_diag ? g - tic * (tic - 1) / 2 : g - tic * (tic + 1) / 2;
        if (int(threadIdx.x) < NSLOT) {
          int64_t ti = tic, tj = tjc;
#pragma unroll
          for (int l = 0; l < H; ++l) { ti = ins0(ti, d.hpos[l]); tj = ins0(tj, d.hpos[l]); }
          const int x = int(threadIdx.x) >> H, y = int(threadIdx.x) & (S - 1);
#pragma unroll
          for (int l = 0; l < H; ++l) {
            ti |= int64_t((x >> l) & 1) << d.hpos[l];
            tj |= int64_t((y >> l) & 1) << d.hpos[l];
          }
          t = ti < tj;
          v = true;
          s_base[b][threadIdx.x] = (t ? tj * (tj + 1) / 2 + ti : ti * (ti + 1) / 2 + tj) * tile_elems;
        }
      }
      const unsigned tmask = __ballot_sync(0xffffffffu, t);
      const unsigned vmask = __ballot_sync(0xffffffffu, v);
      if (threadIdx.x == 0) {
        s_tmask[b] = tmask;
        s_vmask[b] = vmask;
        s_diag[b] = !PACK && (tic == tjc);
      }
    }
  };
  // Asynchronous loads of item w into stage buffer `buf`: rows of lower slots as
  // 16-byte granules; upper slots element by element into their transposed
  // (logical) place, reading the stored partner along its rows.
  // 16-byte elements in slots smaller than the CTA (two high qubits at m = 5,
  // and m <= 4): one flat walk over the item's elements, the slot's
  // transposed bit selecting the shared and global addresses (a lower slot is
  // read along its rows into place, an upper one along its stored rows into
  // the transposed place).  A per-slot loop there leaves threads idle in every
  // slot and branches per slot; with slots of at least kMainThreads elements
  // the per-slot loop issues fewer instructions than the flat walk's selects.
  constexpr bool FLAT = GSH == 0 && (1 << slot_log2) < kMainThreads;
  // 8-byte elements: the same flat walk over 16-byte granules for items whose
  // slots are all lower (every item of a row-chunked pass, whose diagonal
  // groups run in pass_kernel_diag), when a slot has fewer granules than the CTA
  constexpr int GSL = slot_log2 - GSH;   // log2 granules per slot
  constexpr bool FLATG = GSH == 1 && (1 << GSL) < kMainThreads;
  constexpr int TOTG = NSLOT << GSL;
  constexpr int KG = (TOTG + kMainThreads - 1) / kMainThreads;
  constexpr int TOT = NSLOT << slot_log2;
  constexpr int KF = (TOT + kMainThreads - 1) / kMainThreads;
  auto flat = [&](int f, int& slot, int& srow, int& scol, int& goff, int r0, unsigned tm) {
    slot = f >> slot_log2;
    const int within = f & ((1 << slot_log2) - 1);
    const bool t = (tm >> slot) & 1u;
    srow = t ? (within & (R - 1)) : (within >> m);
    scol = t ? (within >> rl) : (within & (M - 1));
    goff = t ? (scol * M + r0 + srow) : ((r0 + srow) * M + scol);
  };
  auto issue_loads = [&](int64_t w, int b, E* buf) {
    const int r0 = int(w & chunk_mask) << rl;
    const unsigned tm = s_tmask[b], vm = s_vmask[b];
    if constexpr (FLAT) {
#pragma unroll
      for (int k = 0; k < KF; ++k) {
        const int f = int(threadIdx.x) + k * kMainThreads;
        if (TOT % kMainThreads == 0 || f < TOT) {
          int slot, srow, scol, goff;
          flat(f, slot, srow, scol, goff, r0, tm);
          if ((vm >> slot) & 1u)
            cp_async16(buf + (slot << slot_log2) + (srow << m) + (scol ^ G::swz(srow)), st + s_base[b][slot] + goff);
        }
      }
      return;
    }
    if constexpr (FLATG) {
      if (tm == 0u) {
#pragma unroll
        for (int k = 0; k < KG; ++k) {
          const int g = int(threadIdx.x) + k * kMainThreads;
          if (TOTG % kMainThreads == 0 || g < TOTG) {
            const int slot = g >> GSL, within = (g & ((1 << GSL) - 1)) << GSH;
            const int pr = within >> m, pc = within & (M - 1);
            if ((vm >> slot) & 1u)
              cp_async16(buf + (slot << slot_log2) + (pr << m) + (pc ^ G::swz(pr)), st + s_base[b][slot] + (r0 + pr) * M + pc);
          }
        }
        return;
      }
    }
#pragma unroll 1
    for (int slot = 0; slot < NSLOT; ++slot) {
      if (!((vm >> slot) & 1u)) continue;
      const E* gbase = st + s_base[b][slot];
      E* sbuf = buf + (slot << slot_log2);
      if (!((tm >> slot) & 1u)) {
        constexpr int NG = 1 << (slot_log2 - GSH);
#pragma unroll
        for (int k = 0; k < (NG + kMainThreads - 1) / kMainThreads; ++k) {
          const int g = int(threadIdx.x) + k * kMainThreads;
          if (NG % kMainThreads == 0 || g < NG) {
            const int within = g << GSH;
            const int pr = within >> m, pc = within & (M - 1);
            cp_async16(sbuf + (pr << m) + (pc ^ G::swz(pr)), gbase + (r0 + pr) * M + pc);
          }
        }
      } else {
        constexpr int NE = 1 << slot_log2;
#pragma unroll
        for (int k = 0; k < (NE + kMainThreads - 1) / kMainThreads; ++k) {
          const int e = int(threadIdx.x) + k * kMainThreads;
          if (NE % kMainThreads == 0 || e < NE) {
            const int sr = e >> rl, sc = e & (R - 1);   // stored row / column (within the chunk)
            cp_async_elem(sbuf + (sc << m) + (sr ^ G::swz(sc)), gbase + sr * M + r0 + sc);
          }
        }
      }
    }
  };

  // Three stages, two items of copies in flight: item i computes in buffer
  // i % 3 while the copies of items i + 1 and i + 2 fill the other two.  The
  // copies of item i + 2 are issued after the barrier that ends item i - 1,
  // whose buffer they reuse; slot info runs one item further ahead (item i + 3
  // is decoded meanwhile and made visible by the barriers that follow).
  const int64_t G0 = gridDim.x;
  int64_t w = blockIdx.x;
  for (int k = 0; k < 3; ++k)
    if (w + k * G0 < d.n_items) item_info(w + k * G0, k);
  __syncthreads();
  for (int k = 0; k < 2; ++k) {
    if (w + k * G0 < d.n_items) issue_loads(w + k * G0, k, bufs + k * buf_elems);
    cp_async_commit();
  }
  for (int it = 0; w < d.n_items; ++it, w += G0) {
    const int ic = it % 3, ii = it & 3;
    E* sm = bufs + ic * buf_elems;
    cp_async_wait_prev();   // the copies of item it are done (item it + 1 may still be in flight)
    __syncthreads();        // ... and visible; every thread is past item it - 1
    if (w + 2 * G0 < d.n_items) issue_loads(w + 2 * G0, (it + 2) & 3, bufs + ((it + 2) % 3) * buf_elems);
    cp_async_commit();
    if (w + 3 * G0 < d.n_items) item_info(w + 3 * G0, (it + 3) & 3);

    const unsigned tm = s_tmask[ii], vm = s_vmask[ii];
    if (tm) {   // upper slots arrive transposed but not yet conjugated
      if constexpr (FLAT) {
#pragma unroll
        for (int k = 0; k < KF; ++k) {
          const int f = int(threadIdx.x) + k * kMainThreads;
          if ((TOT % kMainThreads == 0 || f < TOT) && ((tm >> (f >> slot_log2)) & 1u)) sm[f] = P::conj_if(sm[f], 1u);
        }
      } else {
#pragma unroll 1
      for (int slot = 0; slot < NSLOT; ++slot) {
        if (!((tm >> slot) & 1u)) continue;
        E* sbuf = sm + (slot << slot_log2);
#pragma unroll
        for (int k = 0; k < ((1 << slot_log2) + kMainThreads - 1) / kMainThreads; ++k) {
          const int e = int(threadIdx.x) + k * kMainThreads;
          if ((1 << slot_log2) % kMainThreads == 0 || e < (1 << slot_log2)) sbuf[e] = P::conj_if(sbuf[e], 1u);
        }
      }
      }
      __syncthreads();
    }
    for (int o = 0; o < d.nops; ++o) {
      const PassOp& op = d.ops[o];
      if (op.nq == 1) apply_1q<P, G, kMainThreads, rows_log2g, cols_log2g, P2>(sm, gm, op, d.coef);
      else if (!P2 || op.kind == OP_U2 || op.kind == OP_MONO2)
        apply_u2_sep<P, G, kMainThreads, rows_log2g, cols_log2g, P2>(sm, gm, op, d.coef);
      else if constexpr (P2) apply_ptm2<P, G, kMainThreads, rows_log2g, cols_log2g>(sm, gm, op, d.coef);
      __syncthreads();
    }
    // write back, each stored tile exactly once: lower slots as 16-byte row
    // granules, upper slots conjugated into their stored partner (skipped in
    // a diagonal group, where they mirror lower slots of the same group)
    const int r0 = int(w & chunk_mask) << rl;
    const bool diag = s_diag[ii];
    if constexpr (FLAT) {
      // an upper slot goes back conjugated into its stored partner, except in
      // a diagonal group (there it mirrors a lower slot of the same group)
      const unsigned wm = vm & (diag ? ~tm : ~0u);
#pragma unroll
      for (int k = 0; k < KF; ++k) {
        const int f = int(threadIdx.x) + k * kMainThreads;
        if (TOT % kMainThreads == 0 || f < TOT) {
          int slot, srow, scol, goff;
          flat(f, slot, srow, scol, goff, r0, tm);
          if ((wm >> slot) & 1u)
            st[s_base[ii][slot] + goff] =
                P::conj_if(sm[(slot << slot_log2) + (srow << m) + (scol ^ G::swz(srow))], (tm >> slot) & 1u);
        }
      }
      continue;
    }
    if constexpr (FLATG) {
      if (tm == 0u) {
#pragma unroll
        for (int k = 0; k < KG; ++k) {
          const int g = int(threadIdx.x) + k * kMainThreads;
          if (TOTG % kMainThreads == 0 || g < TOTG) {
            const int slot = g >> GSL, within = (g & ((1 << GSL) - 1)) << GSH;
            const int pr = within >> m, pc = within & (M - 1);
            if ((vm >> slot) & 1u)
              *reinterpret_cast<uint4*>(st + s_base[ii][slot] + (r0 + pr) * M + pc) =
                  *reinterpret_cast<const uint4*>(sm + (slot << slot_log2) + (pr << m) + (pc ^ G::swz(pr)));
          }
        }
        continue;
      }
    }
#pragma unroll 1
    for (int slot = 0; slot < NSLOT; ++slot) {
      if (!((vm >> slot) & 1u)) continue;
      E* gbase = st + s_base[ii][slot];
      const E* sbuf = sm + (slot << slot_log2);
      if (!((tm >> slot) & 1u)) {
        constexpr int NG = 1 << (slot_log2 - GSH);
#pragma unroll
        for (int k = 0; k < (NG + kMainThreads - 1) / kMainThreads; ++k) {
          const int g = int(threadIdx.x) + k * kMainThreads;
          if (NG % kMainThreads == 0 || g < NG) {
            const int within = g << GSH;
            const int pr = within >> m, pc = within & (M - 1);
            *reinterpret_cast<uint4*>(gbase + (r0 + pr) * M + pc) =
                *reinterpret_cast<const uint4*>(sbuf + (pr << m) + (pc ^ G::swz(pr)));
          }
        }
      } else if (!diag) {
        constexpr int NE = 1 << slot_log2;
#pragma unroll
        for (int k = 0; k < (NE + kMainThreads - 1) / kMainThreads; ++k) {
          const int e = int(threadIdx.x) + k * kMainThreads;
          if (NE % kMainThreads == 0 || e < NE) {
            const int sr = e >> rl, sc = e & (R - 1);
            gbase[sr * M + r0 + sc] = P::conj_if(sbuf[(sc << m) + (sr ^ G::swz(sc))], 1u);
          }
        }
      }
    }
  }
  cp_async_wait_all();
}

// ------------------------------------------------------------------ diagonal groups
// A diagonal group (ti == tj before the high bits are inserted) is hermitian
// as a whole: of its 2^h x 2^h slots only the S (S + 1) / 2 with x >= y are
// stored, and the slot (y, x) above is the conjugate transpose of (x, y).
// Generalising crossTileDiag (the t_i == t_j subcase of Algorithm 3), this
// kernel keeps just the stored slots (full tile height) in shared memory and
// applies every op to one block of each mirror pair {B, B^T}: elements in an
// upper slot are read and written as conjugates of their stored partner, and
// inside a diagonal slot both (r, c) and (c, r) are written.  Used for the
// passes whose tile groups do not fit shared memory at full height.
struct DMap {
  int m, sw;
  __device__ __forceinline__ int at(int s, int r, int c) const { return (((s << m) | r) << m) | (c ^ (r & sw)); }
};

template <class P>
__device__ __forceinline__ Cx<P> dread(const typename P::Elem* sm, const DMap& mp, int li, int lj) {
  const int M1 = (1 << mp.m) - 1;
  const int x = li >> mp.m, r = li & M1, y = lj >> mp.m, c = lj & M1;
  if (x >= y) {
    const auto e = sm[mp.at(x * (x + 1) / 2 + y, r, c)];
    return Cx<P>{P::re(e), P::im(e)};
  }
  const auto e = sm[mp.at(y * (y + 1) / 2 + x, c, r)];
  return Cx<P>{P::re(e), P::flip(P::im(e))};
}

template <class P>
__device__ __forceinline__ void dwrite(typename P::Elem* sm, const DMap& mp, int li, int lj, const Cx<P>& v) {
  const int M1 = (1 << mp.m) - 1;
  const int x = li >> mp.m, r = li & M1, y = lj >> mp.m, c = lj & M1;
  if (x > y) {
    sm[mp.at(x * (x + 1) / 2 + y, r, c)] = P::make(v.re, v.im);
  } else if (x == y) {
    sm[mp.at(x * (x + 1) / 2 + x, r, c)] = P::make(v.re, v.im);
    if (r != c) sm[mp.at(x * (x + 1) / 2 + x, c, r)] = P::make(v.re, P::flip(v.im));
  } else {
    sm[mp.at(y * (y + 1) / 2 + x, c, r)] = P::make(v.re, P::flip(v.im));
  }
}

template <class P>
__device__ __forceinline__ void diag_apply(typename P::Elem* sm, const DMap& mp, const PassOp& op,
                                           const double* coef, int log2g) {
  // blocks (i, j), i >= j, of the (2^log2g / 2^k)^2 block grid; rows and
  // columns share the bit positions op.cbit (no chunking here)
  const int k = op.nq;
  const int nb1 = 1 << (log2g - k);
  const int nblk = nb1 * (nb1 + 1) / 2;
  const double* cf = coef + op.coef;
  for (int b = threadIdx.x; b < nblk; b += kThreads) {
    const int i = int(tri_row(b)), j = b - i * (i + 1) / 2;
    if (k == 1) {
      const int rb = ins0i(i, op.cbit[0]), cb = ins0i(j, op.cbit[0]), bit = 1 << op.cbit[0];
      Cx<P> a = dread<P>(sm, mp, rb, cb), bb = dread<P>(sm, mp, rb, cb | bit);
      Cx<P> c = dread<P>(sm, mp, rb | bit, cb), d = dread<P>(sm, mp, rb | bit, cb | bit);
      if (op.kind == OP_PTM1_U) body_ptm1_u<P>(a, bb, c, d, cf);
      else if (op.kind == OP_PTM1_AD) body_ptm1_ad<P>(a, bb, c, d, cf);
      else if (op.kind == OP_MONO1) body_mono1<P>(a, bb, c, d, cf);
      else body_ptm1<P>(a, bb, c, d, cf);
      dwrite<P>(sm, mp, rb, cb, a);
      dwrite<P>(sm, mp, rb, cb | bit, bb);
      dwrite<P>(sm, mp, rb | bit, cb, c);
      dwrite<P>(sm, mp, rb | bit, cb | bit, d);
    } else {
      const int rb = ins0i(ins0i(i, op.cbit[0]), op.cbit[1]);
      const int cb = ins0i(ins0i(j, op.cbit[0]), op.cbit[1]);
      int rows[4], cols[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        rows[a] = rb | ((a & 1) << op.cbit[0]) | ((a >> 1) << op.cbit[1]);
        cols[a] = cb | ((a & 1) << op.cbit[0]) | ((a >> 1) << op.cbit[1]);
      }
      Cx<P> h[16];
#pragma unroll
      for (int ra = 0; ra < 4; ++ra)
#pragma unroll
        for (int ca = 0; ca < 4; ++ca) h[4 * ra + ca] = dread<P>(sm, mp, rows[ra], cols[ca]);
      if (op.kind == OP_U2) body_u2<P, false>(h, cf);
      else if (op.kind == OP_MONO2) body_u2<P, true>(h, cf);
      else body_ptm2<P>(h, cf);
#pragma unroll
      for (int ra = 0; ra < 4; ++ra)
#pragma unroll
        for (int ca = 0; ca < 4; ++ca) dwrite<P>(sm, mp, rows[ra], cols[ca], h[4 * ra + ca]);
    }
  }
}

template <class P, int H>
__global__ void __launch_bounds__(kThreads, 1)
pass_kernel_diag(typename P::Elem* __restrict__ st, const __grid_constant__ PassDesc d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto* sm = reinterpret_cast<typename P::Elem*>(smem_raw);
  constexpr int S = 1 << H;
  constexpr int NS = S * (S + 1) / 2;
  const int m = d.m;
  const int M = 1 << m;
  const int64_t tile_elems = int64_t(1) << (2 * m);
  const DMap mp{m, P::kSwizzle & (M - 1)};
  for (int64_t t = blockIdx.x; t < d.nt_c; t += gridDim.x) {
    int64_t b = t;
#pragma unroll
    for (int l = 0; l < H; ++l) b = ins0(b, d.hpos[l]);
    for (int pass = 0; pass < 2; ++pass) {
      // pass 0 loads the stored slots, pass 1 (after the ops) stores them back
      if (pass == 1) {
        for (int o = 0; o < d.nops; ++o) {
          diag_apply<P>(sm, mp, d.ops[o], d.coef, H + m);
          __syncthreads();
        }
      }
#pragma unroll 4
      for (int e = threadIdx.x; e < (NS << (2 * m)); e += kThreads) {
        const int s = e >> (2 * m);
        const int w = e & ((1 << (2 * m)) - 1);
        const int x = int(tri_row(s)), y = s - x * (x + 1) / 2;
        int64_t ti = b, tj = b;
#pragma unroll
        for (int l = 0; l < H; ++l) {
          ti |= int64_t((x >> l) & 1) << d.hpos[l];
          tj |= int64_t((y >> l) & 1) << d.hpos[l];
        }
        const int r = w >> m, c = w & (M - 1);
        const int64_t off = (ti * (ti + 1) / 2 + tj) * tile_elems + w;
        if (pass == 0) sm[mp.at(s, r, c)] = st[off];
        else st[off] = sm[mp.at(s, r, c)];
      }
      __syncthreads();
    }
  }
}

// Occupancy-sized persistent grid for one kernel instantiation (cached per device and smem size).
struct LaunchCache {
  int dev = -1;
  size_t smem = 0;
  int blocks = 0;
  int sms = 0;
};

template <class E>
cudaError_t launch_one(void (*kfn)(E*, PassDesc), LaunchCache& lc, int threads, size_t smem, int64_t items,
                       void* state, const PassDesc& d, cudaStream_t s) {
  if (items <= 0) return cudaSuccess;
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (lc.dev != dev || lc.smem != smem) {
    err = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (err != cudaSuccess) return err;
    int nb = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kfn, threads, smem);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&lc.sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    lc.dev = dev;
    lc.smem = smem;
    lc.blocks = nb > 0 ? nb : 1;
  }
  int64_t grid = int64_t(lc.blocks) * lc.sms;
  if (grid > items) grid = items;
  kfn<<<dim3(unsigned(grid)), dim3(threads), smem, s>>>(reinterpret_cast<E*>(state), d);
  return cudaGetLastError();
}

template <class P, int H, int MLOG, bool P2>
cudaError_t launch_t(void* state, const PassDesc& d, cudaStream_t s, int* launches) {
  using E = typename P::Elem;
  constexpr int S_DIAG = (1 << H) * ((1 << H) + 1) / 2;   // stored slots of a diagonal group
  // in-tile passes run packed on the one-high-qubit geometry (four tiles per item)
  constexpr int HK = H == 0 ? 1 : H;
  constexpr int RL = rows_log2_ct(HK, MLOG, int(sizeof(E)));
  if (d.rows_log2 != RL || d.m != MLOG) return cudaErrorInvalidValue;
  static thread_local LaunchCache main_cache, diag_cache;
  // three pipeline stages of one work item each
  const size_t smem = 3 * sizeof(E) * (size_t(1) << (2 * HK + RL + MLOG));
  cudaError_t err = launch_one<E>(pass_kernel<P, HK, MLOG, H == 0, P2>, main_cache, kMainThreads, smem,
                                  d.n_items, state, d, s);
  if (err != cudaSuccess) return err;
  int n = d.n_items > 0 ? 1 : 0;
  // only two-high-qubit passes are row-chunked (tile_log2 <= 5)
  if constexpr (H == 2) {
    if (d.skip_diag) {
      const size_t dsmem = sizeof(E) * size_t(S_DIAG) * (size_t(1) << (2 * d.m));
      err = launch_one<E>(pass_kernel_diag<P, H>, diag_cache, kThreads, dsmem, d.nt_c, state, d, s);
      if (err != cudaSuccess) return err;
      n += 1;
    }
  } else {
    if (d.skip_diag) return cudaErrorInvalidValue;
  }
  if (launches) *launches = n;
  return cudaSuccess;
}

template <class P, int H, bool P2>
cudaError_t launch_m(void* state, const PassDesc& d, cudaStream_t s, int* launches) {
  switch (d.m) {
    case 3: return launch_t<P, H, 3, P2>(state, d, s, launches);
    case 4: return launch_t<P, H, 4, P2>(state, d, s, launches);
    case 5: return launch_t<P, H, 5, P2>(state, d, s, launches);
  }
  return cudaErrorInvalidValue;
}

template <class P, bool P2>
cudaError_t launch_p(void* state, const PassDesc& d, cudaStream_t s, int* launches) {
  if (launches) *launches = 0;
  switch (d.h) {
    case 0: return launch_m<P, 0, P2>(state, d, s, launches);
    case 1: return launch_m<P, 1, P2>(state, d, s, launches);
    case 2: return launch_m<P, 2, P2>(state, d, s, launches);
  }
  return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace orkan
