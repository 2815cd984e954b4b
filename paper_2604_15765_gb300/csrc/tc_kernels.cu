// Tensor-core conjugation of every stored tile by one composed in-tile block.
//
// A run of consecutive unitaries whose qubits all lie inside the tile (every
// target below m, Sec. III-C's intra-tile case) is, as a whole, one unitary
// L_blk on the tile's m qubits (composed on the host in FP64), and the run
// maps every stored tile T -- diagonal or not -- to L_blk T L_blk^dagger
// (Eq. 2 with k = m).  That is a dense complex contraction, two 32 x 32 x 32
// products per tile at m = 5, independent of the run's length, so it goes to
// the 5th-generation tensor cores:
//
//   GEMM 1 (A = T^T per tile, B = L^T):   Y^T = T^T L^T
//   GEMM 2 (A = conj(Y) per tile, B = L^T): conj(T') = conj(Y) L^T,
//                                          since T' = Y L^dagger
//
// Complex products run as real ones, [Cr Ci] = [Ar Ai] [[Br, Bi], [-Bi, Br]],
// so one CTA step is a 128 x 64 x 64 real GEMM: four tiles (32 rows each) on
// M = 128, real and imaginary parts on N = K = 64.  Both GEMMs share the same
// B.  FP32 accuracy comes from the split-TF32 scheme: a = a_hi + a_lo with
// a_hi = tf32(a), a_lo = tf32(a - a_hi), and A B ~ A_hi B_hi + A_hi B_lo +
// A_lo B_hi (the dropped A_lo B_lo term is below 2^-22 relative).
//
// tcgen05.mma (kind::tf32, cta_group::1, M = 128, N = 64, K = 8 per
// instruction) is issued by one thread; operands are K-major, no swizzle,
// 8-row x 16-byte core matrices (leading byte offset 144 B along K, stride
// byte offset 2304 B between 8-row groups); the FP32 accumulators live in
// TMEM (128 lanes x 64 columns per GEMM) and come back with tcgen05.ld
// 32x32b: 256 threads, thread t reads lane t mod 128 (its warp's lane quarter
// is warp mod 4) and the half t / 128 of the row's index range.  Completion is signalled by tcgen05.commit
// on an mbarrier; every wait on it is bounded and sets an error word instead
// of hanging.  complex64 storage (8-byte elements) at m = 5.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "orkan_internal.h"
#include "device_util.cuh"

namespace orkan {
namespace {

constexpr int kTcThreads = 256;   // two warpgroups: TMEM lane quarter = warp % 4, the halves split the columns
// K-direction core-matrix stride: 144 B instead of the packed 128 B leaves a
// 16-byte gap after each core matrix, which puts the four 32-bit words of K
// core c of row r in banks 4 (c + r) .. 4 (c + r) + 3 (mod 32): a warp storing
// 32 consecutive K indices of one row, or rows 0..7 x 4 K indices, hits 32
// distinct banks.
constexpr uint32_t kLbo = 144;
constexpr uint32_t kSboA = 16 * kLbo;          // 8-row group stride (16 K cores)
constexpr uint32_t kSboB = 16 * kLbo;
constexpr uint32_t kABytes = 16 * kSboA;       // one A operand (hi or lo), 128 rows: 36 KiB
constexpr uint32_t kBBytes = 8 * kSboB;        // one B operand, 64 rows: 18 KiB
constexpr uint32_t kSmemBytes = 2 * kABytes + 2 * kBBytes;   // 108 KiB
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(64 >> 3) << 17) | (uint32_t(128 >> 4) << 24);
constexpr long long kWaitLimit = 1 << 24;      // polls of one mbarrier phase before giving up
constexpr uint32_t kOutRow = 272;              // padded byte stride of a staged output row
static_assert(128 * kOutRow <= kABytes, "output staging fits the A_hi buffer");

__device__ __forceinline__ uint32_t saddr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t sbo) {
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((kLbo >> 4) & 0x3FFF) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}

// Byte offset of element (row, k) of a K-major operand (k < 64).
__device__ __forceinline__ uint32_t koff(int row, int k, uint32_t sbo) {
  return uint32_t(row >> 3) * sbo + uint32_t(k >> 2) * kLbo + uint32_t(row & 7) * 16 + uint32_t(k & 3) * 4;
}

__device__ __forceinline__ float tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// a -> (hi, lo) stored at byte offset off of the hi and lo operand buffers.
__device__ __forceinline__ void put_split(unsigned char* hi, unsigned char* lo, uint32_t off, float a) {
  const float h = tf32(a);
  *reinterpret_cast<float*>(hi + off) = h;
  *reinterpret_cast<float*>(lo + off) = a - h;   // the MMA reads the TF32 part of the low word
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
               :: "r"(d_tmem), "l"(da), "l"(db), "r"(kIdesc), "r"(acc));
}

// D = A_hi B_hi + A_hi B_lo + A_lo B_hi over K = 64 (8 steps of K = 8).
__device__ __forceinline__ void issue_gemm(uint32_t d_tmem, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                           uint32_t b_lo, uint32_t mbar) {
  uint32_t acc = 0;
  for (int kk = 0; kk < 8; ++kk) {
    const uint32_t ko = uint32_t(kk) * 2 * kLbo;
    mma_tf32(d_tmem, sdesc(a_hi + ko, kSboA), sdesc(b_hi + ko, kSboB), acc);
    acc = 1;
    mma_tf32(d_tmem, sdesc(a_hi + ko, kSboA), sdesc(b_lo + ko, kSboB), 1);
    mma_tf32(d_tmem, sdesc(a_lo + ko, kSboA), sdesc(b_hi + ko, kSboB), 1);
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar));
}

// Bounded wait for the given phase parity; false when the limit ran out.
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity) {
  for (long long it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(mbar), "r"(parity));
    if (done) return true;
  }
  return false;
}

// 16 FP32 accumulator columns of this thread's TMEM lane, from column address taddr.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__global__ void __launch_bounds__(kTcThreads, 2) tc_kernel(float2* __restrict__ st, const __grid_constant__ TcDesc d) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* a_hi = sm;
  unsigned char* a_lo = sm + kABytes;
  unsigned char* b_hi = sm + 2 * kABytes;
  unsigned char* b_lo = b_hi + kBBytes;
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t mbar;
  const int t = threadIdx.x;
  // B = [[Re L^T, Im L^T], [-Im L^T, Re L^T]] (64 x 64), element (k, n) on row n of the K-major operand
  for (int i = t; i < 64 * 64; i += kTcThreads) {
    const int k = i >> 6, n = i & 63;
    const float2 l = d.u[(n & 31) * 32 + (k & 31)];   // L^T[k][n] = L[n][k]
    const float v = (k < 32) == (n < 32) ? l.x : (k < 32 ? l.y : -l.y);
    put_split(b_hi, b_lo, koff(n, k, kSboB), v);
  }
  const uint32_t mb = saddr(&mbar);
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (t < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" :: "r"(saddr(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t d1 = tmem_base, d2 = tmem_base + 64;
  const int warp = t >> 5, ln = t & 31;
  const uint32_t lane = uint32_t(32 * (warp & 3)) << 16;   // this warp's TMEM lane quarter
  const uint32_t ah = saddr(a_hi), al = saddr(a_lo), bh = saddr(b_hi), bl = saddr(b_lo);
  const int row = t & 127, half = t >> 7;               // accumulator row (tile tt, column / row c) and half
  const int tt = row >> 5, c = row & 31;
  const int n0 = 16 * half;                             // this thread's 16 of the 32 row / column indices n
  uint32_t parity = 0;
  bool ok = true;
  const int64_t nitems = (d.ntiles + 3) / 4;
  // Load mapping (conflict-free A stores): per step j, tile q, row k and 16-byte
  // column pair cp of the 4 tiles come from (j, warp, lane):
  //   lane = (k & 7) << 2 | (cp & 3), (j, warp) = q, k >> 3, cp >> 2.
  float4 pre[8];
  auto load_item = [&](int64_t it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int h6 = j * 8 + warp;
      const int q = h6 >> 4, k = ((h6 >> 2) & 3) * 8 + (ln >> 2), cp = (h6 & 3) * 4 + (ln & 3);
      const int64_t tile = it * 4 + q;
      pre[j] = tile < d.ntiles ? __ldcs(reinterpret_cast<const float4*>(st + (tile << 10)) + (k * 16 + cp))
                               : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
  };
  // L2 prefetch of an item's four tiles (contiguous 8 KiB each, one bulk
  // prefetch per tile by threads 0..3): issued two items ahead, so the
  // register loads of the next item find their lines in L2
  auto prefetch_item = [&](int64_t it) {
    const int64_t tile = it * 4 + t;
    if (t < 4 && tile < d.ntiles)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], 8192;" :: "l"(st + (tile << 10)) : "memory");
  };
  if (int64_t(blockIdx.x) + gridDim.x < nitems) prefetch_item(blockIdx.x + gridDim.x);
  if (int64_t(blockIdx.x) < nitems) load_item(blockIdx.x);
  for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
    const int64_t tile0 = item * 4;
    // A = T^T: element (k, c) of tile q goes to row 32 q + c, K index k (re) and 32 + k (im)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int h6 = j * 8 + warp;
      const int q = h6 >> 4, k = ((h6 >> 2) & 3) * 8 + (ln >> 2), cc = ((h6 & 3) * 4 + (ln & 3)) * 2;
      put_split(a_hi, a_lo, koff(32 * q + cc, k, kSboA), pre[j].x);
      put_split(a_hi, a_lo, koff(32 * q + cc, 32 + k, kSboA), pre[j].y);
      put_split(a_hi, a_lo, koff(32 * q + cc + 1, k, kSboA), pre[j].z);
      put_split(a_hi, a_lo, koff(32 * q + cc + 1, 32 + k, kSboA), pre[j].w);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (t == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      issue_gemm(d1, ah, al, bh, bl, mb);
    }
    // the next item's tiles stream in while the tensor cores work; the one
    // after it is prefetched into L2
    if (item + gridDim.x < nitems) load_item(item + gridDim.x);
    if (item + 2 * int64_t(gridDim.x) < nitems) prefetch_item(item + 2 * int64_t(gridDim.x));
    ok = __syncthreads_and(wait_phase(mb, parity));
    parity ^= 1;
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;");
    float vr[16], vi[16];
    tmem_ld16(d1 + lane + uint32_t(n0), vr);        // Re Y[n][c], n = n0 .. n0 + 15 (tile tt)
    tmem_ld16(d1 + lane + uint32_t(32 + n0), vi);   // Im Y[n][c]
    // A = conj(Y): row 32 tt + n, K index c (re) and 32 + c (-im); with the
    // 144-byte core stride a warp's 32 K indices land in 32 banks
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      put_split(a_hi, a_lo, koff(32 * tt + n0 + j, c, kSboA), vr[j]);
      put_split(a_hi, a_lo, koff(32 * tt + n0 + j, 32 + c, kSboA), -vi[j]);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (t == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      issue_gemm(d2, ah, al, bh, bl, mb);
    }
    ok = __syncthreads_and(wait_phase(mb, parity));
    parity ^= 1;
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;");
    tmem_ld16(d2 + lane + uint32_t(n0), vr);        // Re conj(T')[c][n] = Re T'[c][n]
    tmem_ld16(d2 + lane + uint32_t(32 + n0), vi);   // Im conj(T')[c][n] = -Im T'[c][n]
    // stage the four output tiles in the (now free) A_hi buffer, rows padded
    // to 272 bytes so a warp's 16-byte stores take four wavefronts, then
    // write them to HBM with each warp covering 512 contiguous bytes per store
    {
      float4* orow = reinterpret_cast<float4*>(a_hi + row * kOutRow + 8 * n0);
#pragma unroll
      for (int j = 0; j < 8; ++j) orow[j] = make_float4(vr[2 * j], -vi[2 * j], vr[2 * j + 1], -vi[2 * j + 1]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int f = j * kTcThreads + t;       // float4 index in the item: tile q, row r, column pair cq
      const int q = f >> 9, r = (f >> 4) & 31, cq = f & 15;
      if (tile0 + q < d.ntiles)
        __stcs(reinterpret_cast<float4*>(st + ((tile0 + q) << 10)) + (f & 511),
               *reinterpret_cast<const float4*>(a_hi + (32 * q + r) * kOutRow + 16 * cq));
    }
    __syncthreads();   // the staged rows are read before the next item's operands overwrite them
  }
  if (!ok) {
    if (t == 0) atomicExch(d.err, 1);
    (void)wait_phase(mb, parity ^ 1);   // bounded: let an MMA still in flight finish before TMEM is freed
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (t < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" :: "r"(tmem_base));
}

}  // namespace

cudaError_t launch_tc(void* state, const TcDesc& d, cudaStream_t s) {
  if (d.ntiles <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemBytes));
  if (err != cudaSuccess) return err;
  // two CTAs per SM (108 KiB of shared memory and 256 x 128 registers each), so
  // that one CTA's tile loads and operand stores overlap the other's MMAs
  const int64_t nitems = (d.ntiles + 3) / 4;
  const int grid = int(std::min<int64_t>(nitems, int64_t(2) * sms));
  tc_kernel<<<grid, kTcThreads, kSmemBytes, s>>>(reinterpret_cast<float2*>(state), d);
  return cudaGetLastError();
}

}  // namespace orkan
