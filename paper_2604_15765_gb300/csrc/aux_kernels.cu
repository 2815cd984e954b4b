// Initialisation, dense export and reductions on the tiled layout.
//
// Layout (Sec. III-B): tile (ti, tj), ti >= tj, starts at element
// (ti (ti + 1) / 2 + tj) M^2; element (r, c) of a tile at r M + c.  Element
// (i, j) with i < j of the operator is the conjugate of (j, i); inside a
// diagonal tile both are stored and the lower one is authoritative.
//
// Reductions accumulate in FP64 for every storage policy (the tiled mean value
// forms its per-tile partial sums of DF64 / C64 products in double-float, see
// TileDot) and are deterministic: a fixed grid of kRedBlocks CTAs, a fixed
// per-thread order, a fixed shuffle tree, and a single-CTA final pass in index
// order.
#include "orkan_internal.h"
#include "numeric.cuh"
#include "device_util.cuh"

namespace orkan {
namespace {

constexpr int kAuxThreads = 256;

template <class P>
__global__ void k_zero(typename P::Elem* st, int64_t count) {
  typename P::Elem z = Conv<P>::from(0.0, 0.0);
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < count; e += int64_t(gridDim.x) * blockDim.x)
    st[e] = z;
}

template <class P>
__global__ void k_set_diag(typename P::Elem* st, int m, int64_t i, double re) {
  const int64_t t = i >> m;
  const int64_t off = tile_base(t, t, m) + (i & ((1 << m) - 1)) * ((int64_t(1) << m) + 1);
  st[off] = Conv<P>::from(re, 0.0);
}

template <class P>
__global__ void k_fill_diag(typename P::Elem* st, int m, int64_t N, double re) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t t = i >> m;
    st[tile_base(t, t, m) + (i & ((1 << m) - 1)) * ((int64_t(1) << m) + 1)] = Conv<P>::from(re, 0.0);
  }
}

// One CTA per stored tile (grid-stride).  mode 0: from a dense row-major
// N x N complex128 matrix; mode 1: from a pure state psi (rho = psi psi^dagger).
template <class P, int MODE>
__global__ void k_from_host(typename P::Elem* st, int m, int64_t N, int64_t ntiles, const double2* src) {
  const int M = 1 << m;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t ti = tri_row(t), tj = t - ti * (ti + 1) / 2;
    const int64_t base = t << (2 * m);
    for (int w = threadIdx.x; w < M * M; w += blockDim.x) {
      const int64_t i = ti * M + (w >> m), j = tj * M + (w & (M - 1));
      double2 v = make_double2(0.0, 0.0);
      if (i < N && j < N) {
        const int64_t a = i >= j ? i : j, b = i >= j ? j : i;   // lower element (a, b)
        if (MODE == 0) {
          v = src[a * N + b];
        } else {
          const double2 pa = src[a], pb = src[b];
          v = make_double2(pa.x * pb.x + pa.y * pb.y, pa.y * pb.x - pa.x * pb.y);
        }
        if (i < j) v.y = -v.y;
      }
      st[base + w] = Conv<P>::from(v.x, v.y);
    }
  }
}

template <class P>
__global__ void k_to_dense(const typename P::Elem* st, int m, int64_t N, int64_t ntiles, double2* dst) {
  const int M = 1 << m;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t ti = tri_row(t), tj = t - ti * (ti + 1) / 2;
    const int64_t base = t << (2 * m);
    for (int w = threadIdx.x; w < M * M; w += blockDim.x) {
      const int64_t i = ti * M + (w >> m), j = tj * M + (w & (M - 1));
      if (i >= N || j >= N || i < j) continue;
      const double2 v = Conv<P>::to(st[base + w]);
      dst[i * N + j] = v;
      if (i != j) dst[j * N + i] = make_double2(v.x, -v.y);
    }
  }
}

template <class P>
__global__ void k_gather(const typename P::Elem* st, int m, int64_t count, const int64_t* rows, const int64_t* cols,
                         double2* out) {
  const int M = 1 << m;
  for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < count; t += int64_t(gridDim.x) * blockDim.x) {
    int64_t i = rows[t], j = cols[t];
    const bool cj = i < j;
    if (cj) { const int64_t x = i; i = j; j = x; }
    double2 v = Conv<P>::to(st[tile_base(i >> m, j >> m, m) + ((i & (M - 1)) << m) + (j & (M - 1))]);
    if (cj) v.y = -v.y;
    out[t] = v;
  }
}

// Pauli-sum observable O = sum_t c_t P_t.  Thread i owns row i of the lower
// triangle: P_t[i, i ^ x_t] = i^{nY} (-1)^{popc(~i & y) + popc(i & z)} (row index
// i; Y contributes -i on a row bit 0 and +i on a row bit 1).  Terms arrive sorted
// by x so that equal x accumulate in FP64 before one conversion per element.
// masks[4 t + {0,1,2,3}] = {x, z, y, nY}.
template <class P>
__global__ void k_pauli_sum(typename P::Elem* st, int m, int64_t N, int nterms, const uint64_t* masks,
                            const double* coeffs) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
    int t = 0;
    while (t < nterms) {
      const uint64_t x = masks[4 * t];
      double re = 0.0, im = 0.0;
      int u = t;
      for (; u < nterms && masks[4 * u] == x; ++u) {
        const uint64_t z = masks[4 * u + 1], y = masks[4 * u + 2];
        const int ny = int(masks[4 * u + 3] & 3);
        const int par = (__popcll(~uint64_t(i) & y) + __popcll(uint64_t(i) & z)) & 1;
        const double s = par ? -coeffs[u] : coeffs[u];
        // multiply s by i^{nY}
        if (ny == 0) re += s;
        else if (ny == 1) im += s;
        else if (ny == 2) re -= s;
        else im -= s;
      }
      const int64_t j = int64_t(uint64_t(i) ^ x);
      if (i >= j) {
        const int64_t off = tile_base(i >> m, j >> m, m) + ((i & ((1 << m) - 1)) << m) + (j & ((1 << m) - 1));
        st[off] = Conv<P>::from(re, im);
        if (i != j && (i >> m) == (j >> m)) {
          // the mirrored element inside a diagonal tile is stored too
          const int64_t off2 = tile_base(i >> m, i >> m, m) + ((j & ((1 << m) - 1)) << m) + (i & ((1 << m) - 1));
          st[off2] = Conv<P>::from(re, -im);
        }
      }
      t = u;
    }
  }
}

// ------------------------------------------------------------------ reductions
template <int K>
__device__ __forceinline__ void block_reduce_store(double (&v)[K], double* out) {
  __shared__ double red[K][kAuxThreads / 32];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int w = 0; w < kAuxThreads / 32; ++w) s += red[k][w];
      out[k] = s;
    }
  }
}

// Final pass: one CTA sums partials[b * K + k] over b in a fixed order.
template <int K>
__global__ void k_finalize(const double* partials, int nblocks, double* res) {
  double v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += partials[b * K + k];
  block_reduce_store<K>(v, res);
}

template <class P>
__global__ void k_reduce_diag(const typename P::Elem* st, int m, int64_t N, int q, double* partials) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t t = i >> m;
    const double2 e = Conv<P>::to(st[tile_base(t, t, m) + (i & ((1 << m) - 1)) * ((int64_t(1) << m) + 1)]);
    v[0] += e.x;
    v[1] += e.y;
    if (q >= 0) {
      if ((i >> q) & 1) v[3] += e.x;
      else v[2] += e.x;
    }
  }
  block_reduce_store<4>(v, partials + 4 * blockIdx.x);
}

template <class P>
__global__ void k_reduce_pauli(const typename P::Elem* st, int m, int64_t N, uint64_t x, uint64_t z, uint64_t y,
                               double* partials) {
  double v[2] = {0.0, 0.0};
  const int M = 1 << m;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t j = int64_t(uint64_t(i) ^ x);   // element h[j, i]
    double2 e;
    if (j >= i) {
      e = Conv<P>::to(st[tile_base(j >> m, i >> m, m) + ((j & (M - 1)) << m) + (i & (M - 1))]);
    } else {
      e = Conv<P>::to(st[tile_base(i >> m, j >> m, m) + ((i & (M - 1)) << m) + (j & (M - 1))]);
      e.y = -e.y;
    }
    const int par = (__popcll(~uint64_t(i) & y) + __popcll(uint64_t(i) & z)) & 1;
    if (par) { v[0] -= e.x; v[1] -= e.y; }
    else { v[0] += e.x; v[1] += e.y; }
  }
  block_reduce_store<2>(v, partials + 2 * blockIdx.x);
}

// a.re b.re + a.im b.im summed over one thread's
// elements of one tile.  C128 accumulates in FP64.  DF64 and C64 form the
// products on the FP32 pipe (TwoProduct of the leading parts plus the cross
// terms) and accumulate them in double-float (TwoSum), converting to FP64 once
// per tile: GB300's FP64 pipe would otherwise bind this HBM-streaming reduction
// (converting every double-float element costs ~14 FP64 operations).
template <class P> struct TileDot;
template <> struct TileDot<PolF64> {
  double s = 0.0;
  __device__ __forceinline__ void add(const double2& a, const double2& b) { s = fma(a.x, b.x, fma(a.y, b.y, s)); }
  __device__ __forceinline__ double get() const { return s; }
};
// Elements (re.hi, im.hi, re.lo, im.lo): the real-part products accumulate in
// lane 0 and the imaginary-part products in lane 1 of one paired sum.
template <> struct TileDot<PolDF64> {
  DF2 acc{make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
  __device__ __forceinline__ void add(const float4& a, const float4& b) {
    acc = df2_mac(acc, DF2{make_float2(a.x, a.y), make_float2(a.z, a.w)},
                  DF2{make_float2(b.x, b.y), make_float2(b.z, b.w)});
  }
  __device__ __forceinline__ double get() const {
    return (double(acc.hi.x) + double(acc.lo.x)) + (double(acc.hi.y) + double(acc.lo.y));
  }
};
template <> struct TileDot<PolF32> {
  DF acc{0.0f, 0.0f};
  __device__ __forceinline__ void add(const float2& a, const float2& b) {
    acc = PolDF64::mac(acc, DF{a.x, 0.0f}, make_float2(b.x, 0.0f));
    acc = PolDF64::mac(acc, DF{a.y, 0.0f}, make_float2(b.y, 0.0f));
  }
  __device__ __forceinline__ double get() const { return double(acc.hi) + double(acc.lo); }
};

template <class P>
__global__ void k_reduce_expect(const typename P::Elem* rho, const typename P::Elem* O, int m, int64_t ntiles,
                                double* partials) {
  double v[1] = {0.0};
  const int MM = 1 << (2 * m);
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t ti = tri_row(t), tj = t - ti * (ti + 1) / 2;
    const int64_t base = t << (2 * m);
    TileDot<P> dot;
    for (int w = threadIdx.x; w < MM; w += blockDim.x) dot.add(rho[base + w], O[base + w]);
    const double s = dot.get();
    v[0] += (ti == tj) ? s : 2.0 * s;
  }
  block_reduce_store<1>(v, partials + blockIdx.x);
}

int grid_for(int64_t work, int per_block = kAuxThreads) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g > 65535LL * 16) g = 65535LL * 16;
  if (g < 1) g = 1;
  return int(g);
}

template <class F>
cudaError_t dispatch(int dtype, F&& f) {
  switch (dtype) {
    case DT_C128: return f(PolF64{});
    case DT_C64: return f(PolF32{});
    case DT_DF64: return f(PolDF64{});
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_zero(int dtype, void* state, const Geometry& g, cudaStream_t s) {
  return dispatch(dtype, [&](auto pol) {
    using P = decltype(pol);
    const int64_t count = g.ntiles << (2 * g.m);
    k_zero<P><<<grid_for(count), kAuxThreads, 0, s>>>(reinterpret_cast<typename P::Elem*>(state), count);
    return cudaGetLastError();
  });
}

cudaError_t launch_set_diag(int dtype, void* state, const Geometry& g, int64_t i, double re, cudaStream_t s) {
  return dispatch(dtype, [&](auto pol) {
    using P = decltype(pol);
    k_set_diag<P><<<1, 1, 0, s>>>(reinterpret_cast<typename P::Elem*>(state), g.m, i, re);
    return cudaGetLastError();
  });
}

cudaError_t launch_fill_diag(int dtype, void* state, const Geometry& g, double re, cudaStream_t s) {
  return dispatch(dtype, [&](auto pol) {
    using P = decltype(pol);
    k_fill_diag<P><<<grid_for(g.N), kAuxThreads, 0, s>>>(reinterpret_cast<typename P::Elem*>(state), g.m, g.N, re);
    return cudaGetLastError();
  });
}

cudaError_t launch_from_dense(int dtype, void* state, const Geometry& g, const double* dense_dev, cudaStream_t s) {
  return dispatch(dtype, [&](auto pol) {
    using P = decltype(pol);
    const int grid = int(g.ntiles < 65535LL * 8 ? g.ntiles : 65535LL * 8);
    k_from_host<P, 0><<<grid, kAuxThreads, 0, s>>>(reinterpret_cast<typename P::Elem*>(state), g.m, g.N, g.ntiles,
                                                   reinterpret_cast<const double2*>(dense_dev));
    return cudaGetLastError();
  });
}

cudaError_t launch_from_pure(int dtype, void* state, const Geometry& g, const double* psi_dev, cudaStream_t s) {
  return dispatch(dtype, [&](auto pol) {
    using P = decltype(pol);
    const int grid = int(g.ntiles < 65535LL * 8 ? g.ntiles : 65535LL * 8);
    k_from_host<P, 1><<<grid, kAuxThreads, 0, s>>>(reinterpret_cast<typename P::Elem*>(state), g.m, g.N, g.ntiles,
                                                   reinterpret_cast<const double2*>(psi_dev));
    return cudaGetLastError();
  });
}

cudaError_t launch_to_dense(int dtype, const void* state, const Geometry& g, double* dense_dev, cudaStream_t s) {
  return dispatch(dtype, [&](auto pol) {
    using P = decltype(pol);
    const int grid = int(g.ntiles < 65535LL * 8 ? g.ntiles : 65535LL * 8);
    k_to_dense<P><<<grid, kAuxThreads, 0, s>>>(reinterpret_cast<const typename P::Elem*>(state), g.m, g.N, g.ntiles,
                                               reinterpret_cast<double2*>(dense_dev));
    return cudaGetLastError();
  });
}

cudaError_t launch_gather(int dtype, const void* state, const Geometry& g, int64_t count, const int64_t* rows_dev,
                          const int64_t* cols_dev, double* out_dev, cudaStream_t s) {
  return dispatch(dtype, [&](auto pol) {
    using P = decltype(pol);
    k_gather<P><<<grid_for(count), kAuxThreads, 0, s>>>(reinterpret_cast<const typename P::Elem*>(state), g.m, count,
                                                        rows_dev, cols_dev, reinterpret_cast<double2*>(out_dev));
    return cudaGetLastError();
  });
}

cudaError_t launch_pauli_sum(int dtype, void* state, const Geometry& g, int nterms, const uint64_t* masks_dev,
                             const double* coeffs_dev, cudaStream_t s) {
  return dispatch(dtype, [&](auto pol) {
    using P = decltype(pol);
    k_pauli_sum<P><<<grid_for(g.N), kAuxThreads, 0, s>>>(reinterpret_cast<typename P::Elem*>(state), g.m, g.N,
                                                         nterms, masks_dev, coeffs_dev);
    return cudaGetLastError();
  });
}

cudaError_t launch_reduce_diag(int dtype, const void* state, const Geometry& g, int q, double* partials,
                               double* res, cudaStream_t s) {
  return dispatch(dtype, [&](auto pol) {
    using P = decltype(pol);
    k_reduce_diag<P><<<kRedBlocks, kAuxThreads, 0, s>>>(reinterpret_cast<const typename P::Elem*>(state), g.m, g.N,
                                                        q, partials);
    k_finalize<4><<<1, kAuxThreads, 0, s>>>(partials, kRedBlocks, res);
    return cudaGetLastError();
  });
}

cudaError_t launch_reduce_pauli(int dtype, const void* state, const Geometry& g, uint64_t xmask, uint64_t zmask,
                                uint64_t ymask, double* partials, double* res, cudaStream_t s) {
  return dispatch(dtype, [&](auto pol) {
    using P = decltype(pol);
    k_reduce_pauli<P><<<kRedBlocks, kAuxThreads, 0, s>>>(reinterpret_cast<const typename P::Elem*>(state), g.m,
                                                         g.N, xmask, zmask, ymask, partials);
    k_finalize<2><<<1, kAuxThreads, 0, s>>>(partials, kRedBlocks, res);
    return cudaGetLastError();
  });
}

cudaError_t launch_reduce_expect(int dtype, const void* rho, const void* O, const Geometry& g, double* partials,
                                 double* res, cudaStream_t s) {
  return dispatch(dtype, [&](auto pol) {
    using P = decltype(pol);
    k_reduce_expect<P><<<kRedBlocks, kAuxThreads, 0, s>>>(reinterpret_cast<const typename P::Elem*>(rho),
                                                          reinterpret_cast<const typename P::Elem*>(O), g.m,
                                                          g.ntiles, partials);
    k_finalize<1><<<1, kAuxThreads, 0, s>>>(partials, kRedBlocks, res);
    return cudaGetLastError();
  });
}

}  // namespace orkan
