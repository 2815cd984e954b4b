// The packed column-major layout (Sec. III-A): the N (N + 1) / 2 lower-triangle
// elements column by column, h_ij (i >= j) at  j N - j (j - 1) / 2 + (i - j).
//
// The library keeps this layout as the comparison point for the tiled one (the
// paper's own benchmarks compare the two).  On the GPU it is implemented the
// natural way for this layout, one op per pass, with no shared-memory staging:
//
//  * a thread updates one 2^k x 2^k block h_{s,s'} (s >= s'; h_{s',s} is its
//    adjoint) straight from HBM, reading an element above the diagonal as the
//    conjugate of its stored partner (the per-element branch the paper names)
//    and writing it back there; in a diagonal block only x >= y is written;
//  * blocks are enumerated column block by column block, rows innermost, so
//    the loads of a warp run along contiguous stretches of the packed columns
//    j0 and j0 + 2^a (at the column distance of Sec. III-A);
//  * the op bodies are the tiled pass kernels' (same arithmetic per block).
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "orkan_internal.h"
#include "numeric.cuh"
#include "device_util.cuh"
#include "pass_kernels.cuh"

namespace orkan {
namespace {

constexpr int kPkThreads = 256;

__device__ __forceinline__ int64_t pk_col(int64_t j, int64_t N) { return j * N - j * (j - 1) / 2; }

template <class P>
__device__ __forceinline__ Cx<P> pk_read(const typename P::Elem* st, int64_t i, int64_t j, int64_t N) {
  const bool cj = i < j;
  const int64_t p = cj ? j : i, q = cj ? i : j;
  const auto e = P::conj_if(st[pk_col(q, N) + (p - q)], cj ? 1u : 0u);
  return Cx<P>{P::re(e), P::im(e)};
}

template <class P>
__device__ __forceinline__ void pk_write(typename P::Elem* st, int64_t i, int64_t j, int64_t N, const Cx<P>& v) {
  const bool cj = i < j;
  const int64_t p = cj ? j : i, q = cj ? i : j;
  st[pk_col(q, N) + (p - q)] = P::conj_if(P::make(v.re, v.im), cj ? 1u : 0u);
}

// One kernel per (policy, k, op form): the form is a compile-time constant, so
// no other form's arithmetic is ever issued.
template <class P, int K, int FORM>
__global__ void __launch_bounds__(kPkThreads) k_packed_op(typename P::Elem* __restrict__ st,
                                                          const __grid_constant__ PackedDesc d) {
  constexpr int B = 1 << K;
  const int64_t N = d.N;
  const int64_t S = N >> K;
  const int q0 = d.q[0], q1 = d.q[1];
  auto dep = [&](int x) -> int64_t {
    return K == 1 ? int64_t(x) << q0 : (int64_t(x & 1) << q0) | (int64_t(x >> 1) << q1);
  };
  // monomial codes in registers once, outside the loop (p: source index, q: phase)
  int pc[B] = {}, qc[B] = {};
  if constexpr (FORM == OP_MONO1 || FORM == OP_MONO2) {
    constexpr int cb = K == 1 ? 0 : 32;
#pragma unroll
    for (int x = 0; x < B; ++x) {
      pc[x] = icoef(d.coef, cb + x);
      qc[x] = icoef(d.coef, cb + B + x);
    }
  }
  for (int64_t g = int64_t(blockIdx.x) * kPkThreads + threadIdx.x; g < d.n_blocks;
       g += int64_t(gridDim.x) * kPkThreads) {
    // g -> (column block sp, row block s >= sp): columns from the last one
    // down (column block sp holds S - sp blocks), rows ascending inside
    const int64_t cr = tri_row(g);
    const int64_t sp = S - 1 - cr;
    const int64_t s = sp + (g - cr * (cr + 1) / 2);
    int64_t ib = ins0(s, q0), jb = ins0(sp, q0);
    if (K == 2) {
      ib = ins0(ib, q1);
      jb = ins0(jb, q1);
    }
    Cx<P> h[B * B];
    const double* cf = d.coef;
    if constexpr (FORM == OP_MONO1) {
      // V[x][p_x] = i^{q_x}: (V h V^dagger)[x][y] = i^{q_x - q_y} h[p_x][p_y];
      // the block is read in its natural order and permuted in registers
      Cx<P> v[4];
#pragma unroll
      for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) v[x * 2 + y] = pk_read<P>(st, ib | dep(x), jb | dep(y), N);
#pragma unroll
      for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
          const int t = pc[x] * 2 + pc[y];
          const Cx<P> z = t == 0 ? v[0] : (t == 1 ? v[1] : (t == 2 ? v[2] : v[3]));
          h[x * 2 + y] = rot_i<P>(z, qc[x] - qc[y]);
        }
    } else if constexpr (FORM == OP_MONO2) {
      // the same permutation for 4x4 blocks, gathered in permuted order
#pragma unroll
      for (int x = 0; x < B; ++x)
#pragma unroll
        for (int y = 0; y < B; ++y)
          h[x * B + y] = rot_i<P>(pk_read<P>(st, ib | dep(pc[x]), jb | dep(pc[y]), N), qc[x] - qc[y]);
    } else {
#pragma unroll
      for (int x = 0; x < B; ++x)
#pragma unroll
        for (int y = 0; y < B; ++y) h[x * B + y] = pk_read<P>(st, ib | dep(x), jb | dep(y), N);
      if constexpr (FORM == OP_PTM1_U) body_ptm1_u<P>(h[0], h[1], h[2], h[3], cf);
      else if constexpr (FORM == OP_PTM1_AD) body_ptm1_ad<P>(h[0], h[1], h[2], h[3], cf);
      else if constexpr (FORM == OP_PTM1) body_ptm1<P>(h[0], h[1], h[2], h[3], cf);
      else body_u2<P, false>(h, cf);
    }
    const bool dblk = s == sp;
#pragma unroll
    for (int x = 0; x < B; ++x)
#pragma unroll
      for (int y = 0; y < B; ++y)
        if (!dblk || x >= y) pk_write<P>(st, ib | dep(x), jb | dep(y), N, h[x * B + y]);
  }
}

// Tiled <-> packed, one thread per stored tiled element.  To packed: the lower
// triangle of every tile (the upper half of diagonal tiles and the padding are
// skipped).  To tiled: every stored element, upper halves of diagonal tiles as
// conjugates, padding as zero.
template <class P>
__global__ void __launch_bounds__(kPkThreads) k_packed_convert(typename P::Elem* __restrict__ packed,
                                                               typename P::Elem* __restrict__ tiled, int m,
                                                               int64_t N, int64_t total, int to_packed) {
  const int M1 = (1 << m) - 1;
  for (int64_t e = int64_t(blockIdx.x) * kPkThreads + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * kPkThreads) {
    const int64_t t = e >> (2 * m);
    const int64_t ti = tri_row(t), tj = t - ti * (ti + 1) / 2;
    const int64_t i = (ti << m) | ((e >> m) & M1), j = (tj << m) | (e & M1);
    const bool active = i < N && j < N;
    if (to_packed) {
      if (active && i >= j) packed[pk_col(j, N) + (i - j)] = tiled[e];
    } else {
      typename P::Elem v = Conv<P>::from(0.0, 0.0);
      if (active) {
        const auto c = pk_read<P>(packed, i, j, N);
        v = P::make(c.re, c.im);
      }
      tiled[e] = v;
    }
  }
}

int grid_for(int64_t work) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 152;
  return int(std::max<int64_t>(1, std::min<int64_t>((work + kPkThreads - 1) / kPkThreads, int64_t(sms) * 16)));
}

template <class P>
cudaError_t launch_packed_t(void* state, const PackedDesc& d, cudaStream_t s) {
  auto* st = reinterpret_cast<typename P::Elem*>(state);
  const int grid = grid_for(d.n_blocks);
  switch (d.kind) {
    case OP_PTM1: k_packed_op<P, 1, OP_PTM1><<<grid, kPkThreads, 0, s>>>(st, d); break;
    case OP_PTM1_U: k_packed_op<P, 1, OP_PTM1_U><<<grid, kPkThreads, 0, s>>>(st, d); break;
    case OP_PTM1_AD: k_packed_op<P, 1, OP_PTM1_AD><<<grid, kPkThreads, 0, s>>>(st, d); break;
    case OP_MONO1: k_packed_op<P, 1, OP_MONO1><<<grid, kPkThreads, 0, s>>>(st, d); break;
    case OP_U2: k_packed_op<P, 2, OP_U2><<<grid, kPkThreads, 0, s>>>(st, d); break;
    case OP_MONO2: k_packed_op<P, 2, OP_MONO2><<<grid, kPkThreads, 0, s>>>(st, d); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class P>
cudaError_t launch_convert_t(void* packed, void* tiled, const Geometry& g, int to_packed, cudaStream_t s) {
  const int64_t total = g.ntiles << (2 * g.m);
  k_packed_convert<P><<<grid_for(total), kPkThreads, 0, s>>>(reinterpret_cast<typename P::Elem*>(packed),
                                                             reinterpret_cast<typename P::Elem*>(tiled), g.m,
                                                             int64_t(1) << g.n, total, to_packed);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_packed(int dtype, void* state, const PackedDesc& d, cudaStream_t stream) {
  if (d.n_blocks <= 0) return cudaSuccess;
  switch (dtype) {
    case DT_C128: return launch_packed_t<PolF64>(state, d, stream);
    case DT_C64: return launch_packed_t<PolF32>(state, d, stream);
    default: return launch_packed_t<PolDF64>(state, d, stream);
  }
}

cudaError_t launch_packed_convert(int dtype, void* packed, void* tiled, const Geometry& g, int to_packed,
                                  cudaStream_t stream) {
  switch (dtype) {
    case DT_C128: return launch_convert_t<PolF64>(packed, tiled, g, to_packed, stream);
    case DT_C64: return launch_convert_t<PolF32>(packed, tiled, g, to_packed, stream);
    default: return launch_convert_t<PolDF64>(packed, tiled, g, to_packed, stream);
  }
}

}  // namespace orkan
