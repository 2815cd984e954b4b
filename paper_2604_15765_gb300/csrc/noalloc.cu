// Pauli-string expectations without any device allocation.
//
// Some callers of this library cannot call cudaMalloc: code that runs while a
// host framework owns all device memory through its own pool (and forbids
// side allocations), code inside latency-critical serving loops where an
// allocation may synchronise the device or fail under fragmentation, and
// plugins that are only handed a device pointer to the tiled operator.  For
// them this file offers one entry point that needs no memory beyond what the
// caller passes in: its scratch space (the per-CTA partial sums of the
// reduction and the per-string results) is a file-scope __device__ array of
// fixed size, so every GPU that loads this library holds it until the process
// exits.
//
// The kernels are a batched copy of the library's Pauli-expectation
// reduction: a fixed grid of kRedBlocks CTAs per string, FP64 accumulation,
// the same per-thread order, shuffle tree and single-CTA final pass, so the
// results equal those of orkan_expect_pauli bit for bit.  The entry point
// sees only a device array, not a handle, so it knows no qubit labels:
// character l of a string acts on physical bit position l of the array.
#include <cstdint>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "../../include/orkan.h"
#include "orkan_internal.h"
#include "numeric.cuh"
#include "device_util.cuh"

namespace orkan {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaMax = ORKAN_NOALLOC_MAX_STRINGS;
constexpr size_t kNaPartials = size_t(kNaMax) * kRedBlocks * 2;   // doubles
constexpr size_t kNaResults = size_t(kNaMax) * 2;                  // doubles

// The shared scratch: partial sums [string][block][re, im], then results [string][re, im].
// Every call writes each partial it later reads, so nothing needs clearing.
static __device__ __align__(256) double g_noalloc_scratch[kNaPartials + kNaResults];

struct PauliBatch {
  uint64_t x[kNaMax];
  uint64_t z[kNaMax];
  uint64_t y[kNaMax];
};

__device__ __forceinline__ void na_block_sum2(double v0, double v1, double* out) {
  __shared__ double red[2][kNaThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_down_sync(0xffffffffu, v0, o);
    v1 += __shfl_down_sync(0xffffffffu, v1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = v0;
    red[1][threadIdx.x >> 5] = v1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < kNaThreads / 32; ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    out[0] = s0;
    out[1] = s1;
  }
}

// blockIdx.y = string; partials[(string * kRedBlocks + block) * 2 + {0, 1}] = sum of sign(i) h[i ^ x, i].
template <class P>
__global__ void k_na_paulis(const typename P::Elem* st, int m, int64_t N, const __grid_constant__ PauliBatch b,
                            double* scratch) {
  const int s = blockIdx.y;
  const uint64_t x = b.x[s], z = b.z[s], y = b.y[s];
  const int M = 1 << m;
  double v0 = 0.0, v1 = 0.0;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t j = int64_t(uint64_t(i) ^ x);
    double2 e;
    if (j >= i) {
      e = Conv<P>::to(st[tile_base(j >> m, i >> m, m) + ((j & (M - 1)) << m) + (i & (M - 1))]);
    } else {
      e = Conv<P>::to(st[tile_base(i >> m, j >> m, m) + ((i & (M - 1)) << m) + (j & (M - 1))]);
      e.y = -e.y;
    }
    const int par = (__popcll(~uint64_t(i) & y) + __popcll(uint64_t(i) & z)) & 1;
    if (par) { v0 -= e.x; v1 -= e.y; }
    else { v0 += e.x; v1 += e.y; }
  }
  na_block_sum2(v0, v1, scratch + (size_t(s) * kRedBlocks + blockIdx.x) * 2);
}

// blockIdx.x = string: results[string] = sum over the string's partials in block order.
__global__ void k_na_finalize(double* scratch) {
  const int s = blockIdx.x;
  const double* part = scratch + size_t(s) * kRedBlocks * 2;
  double v0 = 0.0, v1 = 0.0;
  for (int b = threadIdx.x; b < kRedBlocks; b += blockDim.x) {
    v0 += part[2 * b];
    v1 += part[2 * b + 1];
  }
  na_block_sum2(v0, v1, scratch + kNaPartials + 2 * size_t(s));
}

// Device address of g_noalloc_scratch, looked up once per device (with that
// device current) and kept for the process; it does not survive a
// cudaDeviceReset of that device.
constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
double* g_na_ptr[kMaxDevices] = {};

cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess) return err;
    g_na_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

template <class P>
cudaError_t launch_na(const void* state, int m, int64_t N, int count, const PauliBatch& b, double* scratch,
                      cudaStream_t s) {
  k_na_paulis<P><<<dim3(kRedBlocks, count), kNaThreads, 0, s>>>(reinterpret_cast<const typename P::Elem*>(state),
                                                                m, N, b, scratch);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  k_na_finalize<<<count, kNaThreads, 0, s>>>(scratch);
  return cudaGetLastError();
}

int na_fail(int code, const std::string& msg) {
  set_last_error(msg.c_str());
  return code;
}

}  // namespace
}  // namespace orkan

extern "C" int orkan_expect_paulis_noalloc(const void* dev_state, int n, int dtype, int tile_log2, int count,
                                           const char* paulis, double* out, void* cuda_stream) {
  using namespace orkan;
  if (tile_log2 == 0) tile_log2 = 5;
  if (!dev_state || !paulis || !out) return na_fail(ORKAN_EINVAL, "null argument");
  if (n < 1 || n > 24 || tile_log2 < 3 || tile_log2 > 5 || (dtype != DT_C128 && dtype != DT_C64 && dtype != DT_DF64))
    return na_fail(ORKAN_EINVAL, "bad n / dtype / tile_log2");
  if (count < 1 || count > kNaMax)
    return na_fail(ORKAN_EINVAL, "count must be between 1 and ORKAN_NOALLOC_MAX_STRINGS (" +
                                     std::to_string(kNaMax) + ") strings per call");
  PauliBatch b = {};
  int ny[kNaMax] = {};
  for (int s = 0; s < count; ++s) {
    for (int l = 0; l < n; ++l) {
      const char ch = paulis[size_t(s) * n + l];
      const uint64_t bit = uint64_t(1) << l;
      if (ch == 'I') continue;
      if (ch == 'X') b.x[s] |= bit;
      else if (ch == 'Y') { b.x[s] |= bit; b.y[s] |= bit; ++ny[s]; }
      else if (ch == 'Z') b.z[s] |= bit;
      else return na_fail(ORKAN_EINVAL, "Pauli characters must be I, X, Y or Z");
    }
  }
  double* scratch = nullptr;
  cudaError_t err = scratch_for_current_device(&scratch);
  if (err != cudaSuccess) return na_fail(ORKAN_ECUDA, std::string("scratch set-up: ") + cudaGetErrorString(err));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int64_t N = int64_t(1) << n;
  switch (dtype) {
    case DT_C128: err = launch_na<PolF64>(dev_state, tile_log2, N, count, b, scratch, s); break;
    case DT_C64: err = launch_na<PolF32>(dev_state, tile_log2, N, count, b, scratch, s); break;
    default: err = launch_na<PolDF64>(dev_state, tile_log2, N, count, b, scratch, s); break;
  }
  double res[2 * kNaMax];
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(res, scratch + kNaPartials, sizeof(double) * 2 * count, cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return na_fail(ORKAN_ECUDA, std::string("expect_paulis_noalloc: ") + cudaGetErrorString(err));
  for (int k = 0; k < count; ++k) {
    const double sr = res[2 * k], si = res[2 * k + 1];
    switch (ny[k] & 3) {   // tr(P H) = i^{nY} S
      case 0: out[k] = sr; break;
      case 1: out[k] = -si; break;
      case 2: out[k] = -sr; break;
      default: out[k] = si; break;
    }
  }
  return ORKAN_OK;
}
