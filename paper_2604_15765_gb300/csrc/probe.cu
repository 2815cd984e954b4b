// Pipe-throughput probe of the current GPU: the denominators of the ALU
// rooflines the library reports (FP32 lane operations for the double-float
// and complex64 forms, FP64 operations for complex128).
//
// Each arithmetic kernel runs CH independent dependency chains per thread over
// a fixed number of iterations on 8 CTAs per SM, so that the pipe, not the
// latency of one chain, bounds the rate; the chains feed a guarded store so
// that the compiler keeps them.  The copy kernel moves 16-byte elements with a
// grid-stride loop (read + write bandwidth).
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/orkan.h"
#include "orkan_internal.h"

namespace orkan {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

template <class T, bool FMA>
__global__ void __launch_bounds__(kProbeThreads) k_probe_chain(T* sink, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x) * T(1e-3) + T(c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = FMA ? x[c] * a + b : x[c] + b;
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == T(-1.25)) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true; keeps the chains live
}

// Paired FP32 FMA (f32x2, one instruction for two lanes): CH / 2 chains of
// float2 per thread, the same lane work per iteration as k_probe_chain<float>.
__global__ void __launch_bounds__(kProbeThreads) k_probe_chain2(float* sink, int iters, float a, float b) {
  float2 x[kChains / 2];
#pragma unroll
  for (int c = 0; c < kChains / 2; ++c) x[c] = make_float2(float(threadIdx.x) * 1e-3f + float(c), float(2 * c + 1));
  const float2 aa = make_float2(a, a), bb = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) x[c] = __ffma2_rn(x[c], aa, bb);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains / 2; ++c) s += x[c].x + x[c].y;
  if (s == -1.25f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true; keeps the chains live
}

__global__ void k_probe_copy(const double2* __restrict__ src, double2* __restrict__ dst, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    dst[i] = src[i];
}

template <class K>
float time_ms(K launch, cudaEvent_t e0, cudaEvent_t e1, int reps) {
  launch();
  cudaEventRecord(e0);
  for (int r = 0; r < reps; ++r) launch();
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms / float(reps);
}

}  // namespace
}  // namespace orkan

extern "C" int orkan_probe_pipes(double* out, void* scratch, size_t scratch_bytes) {
  using namespace orkan;
  if (!out || !scratch) {
    set_last_error("null argument");
    return ORKAN_EINVAL;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    set_last_error("no CUDA device");
    return ORKAN_ENODEV;
  }
  const int blocks = sms * 8;
  const size_t sink_bytes = size_t(blocks) * kProbeThreads * sizeof(double);
  // the copy uses two halves of what is left after the sink, in whole 16-byte elements
  const int64_t n = int64_t((scratch_bytes > sink_bytes ? scratch_bytes - sink_bytes : 0) / 32);
  if (n < (int64_t(1) << 20)) {
    set_last_error("scratch too small (needs the sink plus at least 32 MiB)");
    return ORKAN_EINVAL;
  }
  char* base = static_cast<char*>(scratch);
  double* sink = reinterpret_cast<double*>(base);
  double2* src = reinterpret_cast<double2*>(base + sink_bytes);
  double2* dst = src + n;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    set_last_error("cudaEventCreate failed");
    return ORKAN_ECUDA;
  }
  const int iters = 4096;
  const double ops = double(blocks) * kProbeThreads * iters * kChains;
  out[0] = ops / (1e-3 * time_ms([&] { k_probe_chain<float, true><<<blocks, kProbeThreads>>>(
                                       reinterpret_cast<float*>(sink), iters, 1.0000001f, 1e-9f); }, e0, e1, 3));
  out[1] = ops / (1e-3 * time_ms([&] { k_probe_chain<double, true><<<blocks, kProbeThreads>>>(
                                       sink, iters / 16, 1.0000001, 1e-9); }, e0, e1, 3)) / 16.0;
  out[2] = ops / (1e-3 * time_ms([&] { k_probe_chain<float, false><<<blocks, kProbeThreads>>>(
                                       reinterpret_cast<float*>(sink), iters, 1.0f, 1e-9f); }, e0, e1, 3));
  out[3] = ops / (1e-3 * time_ms([&] { k_probe_chain<double, false><<<blocks, kProbeThreads>>>(
                                       sink, iters / 16, 1.0, 1e-9); }, e0, e1, 3)) / 16.0;
  out[5] = ops / (1e-3 * time_ms([&] { k_probe_chain2<<<blocks, kProbeThreads>>>(
                                       reinterpret_cast<float*>(sink), iters, 1.0000001f, 1e-9f); }, e0, e1, 3));
  cudaMemsetAsync(src, 0, size_t(n) * 16);
  out[4] = 2.0 * double(n) * 16.0 /
           (1e-3 * time_ms([&] { k_probe_copy<<<sms * 8, 512>>>(src, dst, n); }, e0, e1, 5)) / 1e9;
  const cudaError_t err = cudaDeviceSynchronize();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) {
    set_last_error(cudaGetErrorString(err));
    return ORKAN_ECUDA;
  }
  return ORKAN_OK;
}
