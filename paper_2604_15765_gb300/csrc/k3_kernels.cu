// Three-qubit operations on the tiled hermitian operator.
//
// Algorithm 1 (Sec. II-A) updates every 2^k x 2^k block h_{s,s'} -- the
// elements whose row and column indices agree with s and s' outside the
// target qubits -- by the Kraus sum of Eq. (2).  With k = 3 a block spans up to
// 2^{2 |A >= m|} = 64 tiles (Sec. III-C), so instead of staging tile groups
// this kernel gathers each block straight from the tiled layout:
//
//  * hermitian ownership: only blocks with s >= s' are updated (h_{s',s} is
//    the adjoint of h_{s,s'}); an element (i, j) with i < j is read as the
//    conjugate of its stored partner (j, i) and written back there, and in a
//    diagonal tile its upper mirror is written as well, so every storage
//    location has exactly one writer;
//  * eight threads per block, thread a holding row a: the row sweep
//    Y = h L^dagger runs in registers, a swizzled shared-memory transpose
//    hands column a of Y to thread a, and the column sweep L Y accumulates
//    the Kraus terms in registers before thread a writes column a back;
//  * monomial unitaries (Toffoli, CCZ, Fredkin, ...) permute the block with
//    quarter-turn phases and no arithmetic.
//
// Consecutive blocks of a row s share s and have consecutive s', so the
// warps' loads of one row i cover contiguous runs of each tile row.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "orkan_internal.h"
#include "numeric.cuh"
#include "device_util.cuh"
#include "pass_kernels.cuh"

namespace orkan {
namespace {

constexpr int kK3Threads = 256;
constexpr int kK3Blocks = kK3Threads / 8;   // 8x8 blocks per CTA and step

// Offset of the stored element holding h[i][j] (lower triangle of the tiled
// layout); cj = true when h[i][j] is the conjugate of the stored value.
__device__ __forceinline__ int64_t k3_loc(uint64_t i, uint64_t j, int m, bool& cj) {
  cj = i < j;
  const uint64_t p = cj ? j : i, q = cj ? i : j;
  const uint64_t M1 = (uint64_t(1) << m) - 1;
  return tile_base(int64_t(p >> m), int64_t(q >> m), m) + int64_t(((p & M1) << m) | (q & M1));
}

template <class P>
__device__ __forceinline__ Cx<P> k3_read(const typename P::Elem* st, uint64_t i, uint64_t j, int m) {
  bool cj;
  const int64_t o = k3_loc(i, j, m, cj);
  const auto e = P::conj_if(st[o], cj ? 1u : 0u);
  return Cx<P>{P::re(e), P::im(e)};
}

// h[i][j] = v: the stored partner, and inside a diagonal tile also the upper mirror.
template <class P>
__device__ __forceinline__ void k3_write(typename P::Elem* st, uint64_t i, uint64_t j, int m, const Cx<P>& v) {
  bool cj;
  const int64_t o = k3_loc(i, j, m, cj);
  const auto e = P::make(v.re, v.im);
  st[o] = P::conj_if(e, cj ? 1u : 0u);
  const uint64_t p = cj ? j : i, q = cj ? i : j;
  if ((p >> m) == (q >> m) && p != q) {
    const uint64_t M1 = (uint64_t(1) << m) - 1;
    st[o - int64_t(((p & M1) << m) | (q & M1)) + int64_t(((q & M1) << m) | (p & M1))] = P::conj_if(e, cj ? 0u : 1u);
  }
}

// One Kraus term on the block row / column of thread a:
// acc[x] (+)= (L (h L^dagger))[x][a], FIRST = start the accumulation.
template <class P, bool FIRST>
__device__ __forceinline__ void k3_term(const Cx<P> (&h)[8], Cx<P> (&acc)[8], typename P::Elem* yb,
                                        const double* cf, int a, unsigned mask) {
  using E = typename P::Elem;
  using R = typename P::Real;
  // row sweep: Y[a][c] = sum_v h[a][v] conj(L[c][v]); one output at a time
  // (each is stored at once), which keeps the register count without spills
#pragma unroll 1
  for (int c = 0; c < 8; ++c) {
    const auto l0r = P::coef(cf, 16 * c), l0i = P::coef(cf, 16 * c + 1);
    R yr = P::mul(h[0].re, l0r);
    yr = P::mac(yr, h[0].im, l0i);
    R yi = P::mul(h[0].im, l0r);
    yi = P::mac(yi, P::neg(h[0].re), l0i);
#pragma unroll
    for (int v = 1; v < 8; ++v) {
      const auto lr = P::coef(cf, 2 * (8 * c + v)), li = P::coef(cf, 2 * (8 * c + v) + 1);
      yr = P::mac(yr, h[v].re, lr);
      yr = P::mac(yr, h[v].im, li);
      yi = P::mac(yi, h[v].im, lr);
      yi = P::mac(yi, P::neg(h[v].re), li);
    }
    yb[(a << 3) | (c ^ a)] = P::make(P::norm(yr), P::norm(yi));
  }
  __syncwarp(mask);
  Cx<P> y[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const E e = yb[(u << 3) | (a ^ u)];
    y[u] = Cx<P>{P::re(e), P::im(e)};
  }
  __syncwarp(mask);   // the next term's row sweep overwrites the staging block
  // column sweep: out[x][a] += sum_u L[x][u] Y[u][a]
#pragma unroll
  for (int x = 0; x < 8; ++x) {
    const auto l0r = P::coef(cf, 16 * x), l0i = P::coef(cf, 16 * x + 1);
    R zr = FIRST ? P::mul(y[0].re, l0r) : P::mac(acc[x].re, y[0].re, l0r);
    R zi = FIRST ? P::mul(y[0].im, l0r) : P::mac(acc[x].im, y[0].im, l0r);
    zr = P::mac(zr, P::neg(y[0].im), l0i);
    zi = P::mac(zi, y[0].re, l0i);
#pragma unroll
    for (int u = 1; u < 8; ++u) {
      const auto lr = P::coef(cf, 2 * (8 * x + u)), li = P::coef(cf, 2 * (8 * x + u) + 1);
      zr = P::mac(zr, y[u].re, lr);
      zr = P::mac(zr, P::neg(y[u].im), li);
      zi = P::mac(zi, y[u].im, lr);
      zi = P::mac(zi, y[u].re, li);
    }
    acc[x] = Cx<P>{P::norm(zr), P::norm(zi)};
  }
}

// MONO: the monomial form (compile-time, so the Kraus sweep carries no codes).
template <class P, bool MONO>
__device__ __forceinline__ void k3_body(typename P::Elem* __restrict__ st, const K3Desc& d) {
  using E = typename P::Elem;
  using R = typename P::Real;
  __shared__ E ybuf[kK3Blocks][64];
  const int a = threadIdx.x & 7;
  const int lb = threadIdx.x >> 3;
  const unsigned mask = 0xffu << (threadIdx.x & 24);   // the 8 lanes of this block
  const int m = d.m;
  const int q0 = d.q[0], q1 = d.q[1], q2 = d.q[2];
  // bits of a local index x placed on the target qubits
  auto dep = [&](int x) -> uint64_t {
    return (uint64_t(x & 1) << q0) | (uint64_t((x >> 1) & 1) << q1) | (uint64_t((x >> 2) & 1) << q2);
  };
  // monomial codes in registers once, outside the loop (p: source index, q:
  // phase).  With 16-byte elements they are packed, 5 bits per local index x
  // (p_x in 3 bits, q_x mod 4 in 2), which keeps the form within the 64
  // registers of four CTAs per SM; 8-byte elements fit there unpacked.
  constexpr bool kPacked = sizeof(typename P::Elem) == 16;
  uint64_t codes = 0;
  int pc[8] = {}, qc[8] = {};
  if constexpr (MONO) {
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      if constexpr (kPacked) {
        codes |= uint64_t((icoef(d.coef, x) & 7) | ((icoef(d.coef, 8 + x) & 3) << 3)) << (5 * x);
      } else {
        pc[x] = icoef(d.coef, x);
        qc[x] = icoef(d.coef, 8 + x);
      }
    }
  }
  auto pcode = [&](int x) { return kPacked ? int(codes >> (5 * x)) & 7 : pc[x]; };
  auto qcode = [&](int x) { return kPacked ? int(codes >> (5 * x + 3)) & 3 : qc[x]; };
  for (int64_t b = int64_t(blockIdx.x) * kK3Blocks + lb; b < d.nblocks; b += int64_t(gridDim.x) * kK3Blocks) {
    const int64_t s = tri_row(b), sp = b - s * (s + 1) / 2;
    const uint64_t ib = uint64_t(ins0(ins0(ins0(s, q0), q1), q2));
    const uint64_t jb = uint64_t(ins0(ins0(ins0(sp, q0), q1), q2));
    const bool dblk = s == sp;   // a hermitian block: only x >= y is written

    if constexpr (MONO) {
      // (L h L^dagger)[a][c] = i^{q_a - q_c} h[p_a][p_c]
      int pa, qa;
      if constexpr (kPacked) {
        pa = pcode(a);
        qa = qcode(a);
      } else {   // select by the runtime lane index without indexing the register arrays
        pa = pc[0];
        qa = qc[0];
#pragma unroll
        for (int x = 1; x < 8; ++x)
          if (a == x) {
            pa = pc[x];
            qa = qc[x];
          }
      }
      const uint64_t isrc = ib | dep(pa);
      Cx<P> v[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) v[c] = rot_i<P>(k3_read<P>(st, isrc, jb | dep(pcode(c)), m), qa - qcode(c));
      __syncwarp(mask);   // every read of the block precedes every write
      const uint64_t i = ib | dep(a);
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (!dblk || a >= c) k3_write<P>(st, i, jb | dep(c), m, v[c]);
    } else {
      Cx<P> h[8];
      {
        const uint64_t i = ib | dep(a);
#pragma unroll
        for (int c = 0; c < 8; ++c) h[c] = k3_read<P>(st, i, jb | dep(c), m);
      }
      Cx<P> acc[8];
      // the first term with compile-time coefficient offsets (the whole of a
      // unitary), further Kraus terms in a loop
      k3_term<P, true>(h, acc, ybuf[lb], d.coef, a, mask);
#pragma unroll 1
      for (int t = 1; t < d.r; ++t) k3_term<P, false>(h, acc, ybuf[lb], d.coef + 128 * t, a, mask);
      const uint64_t j = jb | dep(a);
#pragma unroll
      for (int x = 0; x < 8; ++x)
        if (!dblk || x >= a) k3_write<P>(st, ib | dep(x), j, m, acc[x]);
    }
  }
}

template <class P>
__global__ void __launch_bounds__(kK3Threads) k3_kernel(typename P::Elem* __restrict__ st,
                                                        const __grid_constant__ K3Desc d) {
  k3_body<P, false>(st, d);
}
template <class P>
__global__ void __launch_bounds__(kK3Threads) k3_mono_kernel(typename P::Elem* __restrict__ st,
                                                             const __grid_constant__ K3Desc d) {
  k3_body<P, true>(st, d);
}
// With 16-byte elements the monomial form is held to 64 registers, i.e. four
// CTAs per SM, so that more of its gathers are in flight (8-byte elements fit
// there as they are).
template <class P>
__global__ void __launch_bounds__(kK3Threads, 4) k3_mono4_kernel(typename P::Elem* __restrict__ st,
                                                                 const __grid_constant__ K3Desc d) {
  k3_body<P, true>(st, d);
}

template <class P>
cudaError_t launch_k3_t(void* state, const K3Desc& d, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err != cudaSuccess) return err;
  const int64_t need = (d.nblocks + kK3Blocks - 1) / kK3Blocks;
  const int ctas = int(std::min<int64_t>(need, int64_t(sms) * 8));
  auto* st = reinterpret_cast<typename P::Elem*>(state);
  if (d.form != 1) k3_kernel<P><<<ctas, kK3Threads, 0, s>>>(st, d);
  else if constexpr (sizeof(typename P::Elem) == 16) k3_mono4_kernel<P><<<ctas, kK3Threads, 0, s>>>(st, d);
  else k3_mono_kernel<P><<<ctas, kK3Threads, 0, s>>>(st, d);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_k3(int dtype, void* state, const K3Desc& d, cudaStream_t stream) {
  if (d.nblocks <= 0) return cudaSuccess;
  switch (dtype) {
    case DT_C128: return launch_k3_t<PolF64>(state, d, stream);
    case DT_C64: return launch_k3_t<PolF32>(state, d, stream);
    default: return launch_k3_t<PolDF64>(state, d, stream);
  }
}

}  // namespace orkan
