// Batched circuits: the whole circuits of many small operators in one
// persistent launch.
//
// Each request is one operator in the tiled layout of Sec. III-B with its own
// op list (Eq. 1 / Eq. 2 block updates, Z projections with Born
// renormalisation) and readouts (Pauli-string expectations tr(P H), and
// <psi|H|psi> -- the mean value of Sec. III-C for a pure state).  A small
// operator's per-op pass is far too short to fill a GB300 (a launch costs more
// than the work below n ~ 10), so here CTAs take work slots from a device
// queue (one atomic counter) and each request runs start to end on the CTAs
// that took its slots:
//
//  * gang 1 (operators that fit shared memory, n <= 7): the CTA stages the
//    tiled array in shared memory (or builds it there from the request's
//    initial state), applies every op with a CTA barrier between ops, reads
//    out, and writes the array back once;
//  * gang G > 1 (larger operators): G consecutive slots; the G CTAs split
//    every op's blocks and meet at a gang barrier (an arrival counter in
//    global memory, spun on by one thread with a time limit) between ops.
//    The array stays in global memory (L2-resident at these sizes) and is
//    read and written with L2-coherent loads and stores.
//
// Slots are taken in queue order, so at most one gang is partly taken at any
// time and its missing members are the next slots: with every CTA of the
// grid resident, every gang assembles.  A gang barrier that does not
// complete within the time limit (e.g. a gang larger than the grid) marks its
// request ORKAN_ETIMEOUT and the CTAs move on; nothing waits without a bound.
//
// Block updates follow Algorithm 1 on the tiled layout: every 2^k x 2^k block
// h_{s,s'} with s >= s' (the others are its adjoints), elements above the
// diagonal read as conjugates of their stored partners and written back
// there, and inside a diagonal tile the upper mirror written too, so every
// storage location has exactly one writer per op.  k = 1 ops apply their
// Pauli transfer matrix (Eq. 3 in the Pauli basis, real); k = 2, 3 ops apply
// their Kraus terms as the row sweep h L^dagger and the column sweep L (.).
//
// Every reduction (Born probabilities, readouts) has a fixed order that
// depends only on the request's own n and gang size, so a request's results
// are the same bits alone and in any mix.
#include <type_traits>
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/orkan.h"
#include "orkan_internal.h"
#include "numeric.cuh"
#include "device_util.cuh"

namespace orkan {
namespace {

constexpr int kBT = kBatchThreads;
constexpr int kBW = kBT / 32;

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int64_t bins0(int64_t x, int p) {
  const int64_t low = x & ((int64_t(1) << p) - 1);
  return ((x >> p) << (p + 1)) | low;
}

// Element access at storage offset o of the tiled array: shared memory (gang
// 1) or L2-coherent global accesses (gangs).  In shared memory the FP32-pipe
// forms (complex64, double-float) XOR-permute the element index inside each
// row by a hash of the row counter o >> m (bits 0-2, 3-5, 6-8 and 9-11
// folded), so that the 2^k rows of a block (rows that differ in the target
// bits, inside a tile or across tiles) fall in different 16-byte bank groups;
// the permutation keeps every row in place and is its own inverse.  Native
// FP64 keeps the plain order: there the FP64 pipe binds and the bank
// conflicts hide behind it, so the permutation's integer work would only add
// (measured: 16.6 ms plain vs 16.8 ms permuted for 300 requests of n = 4..8,
// against 12 % less time with the permutation in complex64).
template <class P>
__device__ __forceinline__ int64_t sm_off(int64_t o, int m) {
  if constexpr (std::is_same<typename P::Real, double>::value) {
    return o;
  } else {
    const int64_t x = o >> m;
    return o ^ ((x ^ (x >> 3) ^ (x >> 6) ^ (x >> 9)) & 7);
  }
}
template <class P, bool SM>
struct Acc {
  using E = typename P::Elem;
  static __device__ __forceinline__ E ld(const E* st, int64_t o, int m) {
    if constexpr (SM) return st[sm_off<P>(o, m)];
    else return __ldcg(st + o);
  }
  static __device__ __forceinline__ void st(E* st, int64_t o, int m, const E& v) {
    if constexpr (SM) st[sm_off<P>(o, m)] = v;
    else __stcg(st + o, v);
  }
};

// Storage offset of h[i][j]; cj = the stored value is the conjugate (i < j).
__device__ __forceinline__ int64_t bloc(uint64_t i, uint64_t j, int m, bool& cj) {
  cj = i < j;
  const uint64_t p = cj ? j : i, q = cj ? i : j;
  const uint64_t M1 = (uint64_t(1) << m) - 1;
  return tile_base(int64_t(p >> m), int64_t(q >> m), m) + int64_t(((p & M1) << m) | (q & M1));
}

template <class P, bool SM>
__device__ __forceinline__ Cx<P> bread(const typename P::Elem* st, uint64_t i, uint64_t j, int m) {
  bool cj;
  const int64_t o = bloc(i, j, m, cj);
  const auto e = P::conj_if(Acc<P, SM>::ld(st, o, m), cj ? 1u : 0u);
  return Cx<P>{P::re(e), P::im(e)};
}

template <class P, bool SM>
__device__ __forceinline__ void bwrite(typename P::Elem* st, uint64_t i, uint64_t j, int m, const Cx<P>& v) {
  bool cj;
  const int64_t o = bloc(i, j, m, cj);
  const auto e = P::make(v.re, v.im);
  Acc<P, SM>::st(st, o, m, P::conj_if(e, cj ? 1u : 0u));
  const uint64_t p = cj ? j : i, q = cj ? i : j;
  if ((p >> m) == (q >> m) && p != q) {
    const uint64_t M1 = (uint64_t(1) << m) - 1;
    Acc<P, SM>::st(st, o - int64_t(((p & M1) << m) | (q & M1)) + int64_t(((q & M1) << m) | (p & M1)), m,
                   P::conj_if(e, cj ? 0u : 1u));
  }
}

// A device-side FP64 factor in the policy's coefficient format.
template <class P> __device__ __forceinline__ typename P::Coef dcoef(double v);
template <> __device__ __forceinline__ double dcoef<PolF64>(double v) { return v; }
template <> __device__ __forceinline__ float dcoef<PolF32>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ float2 dcoef<PolDF64>(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}

// Fixed-order CTA sum of K doubles; the totals land in tot[0..K-1] (shared).
template <int K>
__device__ __forceinline__ void cta_sum(double (&v)[K], double* red, double* tot) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[k * kBW + (threadIdx.x >> 5)] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int w = 0; w < kBW; ++w) s += red[k * kBW + w];
      tot[k] = s;
    }
  }
  __syncthreads();
}

struct Ctx {
  const BatchDesc* d;
  const BatchItem* I;
  int it;       // item index
  int g, G;     // rank in the gang, gang size
  int gen;      // barriers passed
};

// Gang barrier: every CTA of the item arrives; returns false when the item
// failed (time limit, or another member marked it), after which the CTA
// leaves the item.  Gang 1: a CTA barrier.
__device__ bool gang_sync(Ctx& c, int* s_flag) {
  __syncthreads();
  if (c.G == 1) return true;
  if (threadIdx.x == 0) {
    int* bar = c.d->bar + c.it;
    int* status = c.d->status + c.it;
    __threadfence();
    atomicAdd(bar, 1);
    const int target = (c.gen + 1) * c.G;
    const uint64_t t0 = now_ns();
    int ok = 1;
    while (ld_acquire(bar) < target) {
      if (ld_acquire(status) != 0) { ok = 0; break; }
      if (now_ns() - t0 > c.d->wait_ns) {
        atomicCAS(status, 0, ORKAN_ETIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    *s_flag = ok;
  }
  __syncthreads();
  ++c.gen;
  return *s_flag != 0;
}

// Sum K per-CTA values over the gang in rank order (FP64); every CTA of the
// gang gets the same totals.  part: this item's gang x stride scratch.
template <int K>
__device__ bool gang_sum(Ctx& c, double (&v)[K], double* red, double* tot, int* s_flag, int slot) {
  cta_sum<K>(v, red, tot);
  if (c.G == 1) return true;
  double* part = c.d->partials + c.I->part_off;
  if (threadIdx.x == 0)
    for (int k = 0; k < K; ++k) __stcg(part + size_t(c.g) * c.I->part_stride + slot + k, tot[k]);
  if (!gang_sync(c, s_flag)) return false;
  if (threadIdx.x == 0)
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int r = 0; r < c.G; ++r) s += __ldcg(part + size_t(r) * c.I->part_stride + slot + k);
      tot[k] = s;
    }
  __syncthreads();
  return true;
}

// Decode storage offset o into the logical pair (i, j) of its element.
__device__ __forceinline__ void decode(int64_t o, int m, uint64_t& i, uint64_t& j) {
  const int64_t t = o >> (2 * m);
  const int64_t ti = tri_row(t), tj = t - ti * (ti + 1) / 2;
  const int64_t M1 = (int64_t(1) << m) - 1;
  i = uint64_t((ti << m) | ((o >> m) & M1));
  j = uint64_t((tj << m) | (o & M1));
}

// ------------------------------------------------------------------ initial operators
template <class P, bool SM>
__device__ void init_pure(const Ctx& c, typename P::Elem* st) {
  const BatchItem& I = *c.I;
  const double2* psi = reinterpret_cast<const double2*>(c.d->aux + I.init_off);
  const uint64_t N = uint64_t(1) << I.n;
  for (int64_t o = int64_t(c.g) * kBT + threadIdx.x; o < I.stored; o += int64_t(c.G) * kBT) {
    uint64_t i, j;
    decode(o, I.m, i, j);
    double re = 0.0, im = 0.0;
    if (i < N && j < N) {
      const double2 a = psi[i], b = psi[j];   // a conj(b)
      re = a.x * b.x + a.y * b.y;
      im = a.y * b.x - a.x * b.y;
    }
    Acc<P, SM>::st(st, o, I.m, Conv<P>::from(re, im));
  }
}

// O[i][j] = sum_t c_t <i|P_t|j>, P_t from masks (x, z, y) with
// <i|P|i^x> = i^{nY} (-1)^{popc(~i & y) + popc(i & z)}.
template <class P, bool SM>
__device__ void init_pauli_sum(const Ctx& c, typename P::Elem* st) {
  const BatchItem& I = *c.I;
  const uint64_t* tm = reinterpret_cast<const uint64_t*>(c.d->aux + I.init_off);
  const double* tc = reinterpret_cast<const double*>(c.d->aux + I.init_off) + 4 * I.nterms;
  const uint64_t N = uint64_t(1) << I.n;
  for (int64_t o = int64_t(c.g) * kBT + threadIdx.x; o < I.stored; o += int64_t(c.G) * kBT) {
    uint64_t i, j;
    decode(o, I.m, i, j);
    double re = 0.0, im = 0.0;
    if (i < N && j < N) {
      for (int t = 0; t < I.nterms; ++t) {
        const uint64_t x = tm[4 * t], z = tm[4 * t + 1], y = tm[4 * t + 2];
        const int ny = int(tm[4 * t + 3]);
        if ((i ^ j) != x) continue;
        double s = ((__popcll(~i & y) + __popcll(i & z)) & 1) ? -tc[t] : tc[t];
        switch (ny & 3) {
          case 0: re += s; break;
          case 1: im += s; break;
          case 2: re -= s; break;
          default: im -= s; break;
        }
      }
    }
    Acc<P, SM>::st(st, o, I.m, Conv<P>::from(re, im));
  }
}

// ------------------------------------------------------------------ k = 1: Pauli transfer matrix
// v = (a + d, b + c, i (b - c), a - d) for the block [[a, b], [c, d]];
// w = (R / 2) v (coefficients prepared on the host); then
// a' = w0 + w3, d' = w0 - w3, b' = w1 - i w2, c' = w1 + i w2.
template <class P, bool SM>
__device__ void apply_ptm1(const Ctx& c, typename P::Elem* st, const BatchOp& op) {
  using R = typename P::Real;
  const BatchItem& I = *c.I;
  const double* cf = c.d->coef + op.coef;
  const int q = op.q[0];
  const int64_t S = int64_t(1) << (I.n - 1);
  const int64_t nb = S * (S + 1) / 2;
  const uint64_t bit = uint64_t(1) << q;
  for (int64_t b = int64_t(c.g) + int64_t(c.G) * threadIdx.x; b < nb; b += int64_t(c.G) * kBT) {
    const int64_t s = tri_row(b), sp = b - s * (s + 1) / 2;
    const uint64_t i0 = uint64_t(bins0(s, q)), j0 = uint64_t(bins0(sp, q));
    const Cx<P> a = bread<P, SM>(st, i0, j0, I.m), bb = bread<P, SM>(st, i0, j0 | bit, I.m);
    const Cx<P> cc = bread<P, SM>(st, i0 | bit, j0, I.m), dd = bread<P, SM>(st, i0 | bit, j0 | bit, I.m);
    R vr[4], vi[4];
    vr[0] = P::add(a.re, dd.re);   vi[0] = P::add(a.im, dd.im);
    vr[1] = P::add(bb.re, cc.re);  vi[1] = P::add(bb.im, cc.im);
    vr[2] = P::sub(cc.im, bb.im);  vi[2] = P::sub(bb.re, cc.re);   // i (b - c)
    vr[3] = P::sub(a.re, dd.re);   vi[3] = P::sub(a.im, dd.im);
    R wr[4], wi[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const auto k0 = P::coef(cf, 4 * x);
      wr[x] = P::mul(vr[0], k0);
      wi[x] = P::mul(vi[0], k0);
#pragma unroll
      for (int y = 1; y < 4; ++y) {
        const auto k = P::coef(cf, 4 * x + y);
        wr[x] = P::mac(wr[x], vr[y], k);
        wi[x] = P::mac(wi[x], vi[y], k);
      }
      wr[x] = P::norm(wr[x]);
      wi[x] = P::norm(wi[x]);
    }
    const Cx<P> na{P::add(wr[0], wr[3]), P::add(wi[0], wi[3])};
    const Cx<P> nd{P::sub(wr[0], wr[3]), P::sub(wi[0], wi[3])};
    const Cx<P> nb_{P::add(wr[1], wi[2]), P::sub(wi[1], wr[2])};   // w1 - i w2
    const Cx<P> nc{P::sub(wr[1], wi[2]), P::add(wi[1], wr[2])};    // w1 + i w2
    bwrite<P, SM>(st, i0, j0, I.m, na);
    bwrite<P, SM>(st, i0 | bit, j0, I.m, nc);
    bwrite<P, SM>(st, i0 | bit, j0 | bit, I.m, nd);
    if (s != sp) bwrite<P, SM>(st, i0, j0 | bit, I.m, nb_);   // in a diagonal block b' is c' mirrored
  }
}

// ------------------------------------------------------------------ k = 2, 3: Kraus sweeps
// D = 2^K lanes per block, lane a holding row a of h_{s,s'}.  Per term:
// Y[a][c] = sum_v h[a][v] conj(L[c][v]) (row sweep), a swizzled transpose
// through shared memory, then out[x][a] += sum_u L[x][u] Y[u][a].
template <class P, bool SM, int K>
__device__ void apply_kraus(const Ctx& c, typename P::Elem* st, const BatchOp& op, typename P::Elem* ybuf) {
  using E = typename P::Elem;
  using R = typename P::Real;
  constexpr int D = 1 << K;
  constexpr int GPC = kBT / D;   // blocks per CTA step
  const BatchItem& I = *c.I;
  const int a = threadIdx.x & (D - 1);
  const int lb = threadIdx.x / D;
  const unsigned mask = ((1u << D) - 1u) << (threadIdx.x & (32 - D));
  E* yb = ybuf + lb * D * D;
  const int q0 = op.q[0], q1 = op.q[1], q2 = op.q[2];
  auto dep = [&](int x) -> uint64_t {
    uint64_t v = (uint64_t(x & 1) << q0) | (uint64_t((x >> 1) & 1) << q1);
    if constexpr (K == 3) v |= uint64_t((x >> 2) & 1) << q2;
    return v;
  };
  auto ins = [&](int64_t s) -> uint64_t {
    int64_t v = bins0(bins0(s, q0), q1);
    if constexpr (K == 3) v = bins0(v, q2);
    return uint64_t(v);
  };
  const int64_t S = int64_t(1) << (I.n - K);
  const int64_t nb = S * (S + 1) / 2;
  const double* cf0 = c.d->coef + op.coef;
  for (int64_t j = lb; ; j += GPC) {
    const int64_t b = int64_t(c.g) + int64_t(c.G) * j;
    if (b >= nb) break;
    const int64_t s = tri_row(b), sp = b - s * (s + 1) / 2;
    const uint64_t ib = ins(s), jb = ins(sp);
    Cx<P> h[D];
#pragma unroll
    for (int v = 0; v < D; ++v) h[v] = bread<P, SM>(st, ib | dep(a), jb | dep(v), I.m);
    Cx<P> acc[D];
#pragma unroll 1
    for (int t = 0; t < op.r; ++t) {
      const double* cf = cf0 + 2 * D * D * t;
#pragma unroll 1
      for (int cc = 0; cc < D; ++cc) {
        R yr = P::mul(h[0].re, P::coef(cf, 2 * D * cc));
        yr = P::mac(yr, h[0].im, P::coef(cf, 2 * D * cc + 1));
        R yi = P::mul(h[0].im, P::coef(cf, 2 * D * cc));
        yi = P::mac(yi, P::neg(h[0].re), P::coef(cf, 2 * D * cc + 1));
#pragma unroll
        for (int v = 1; v < D; ++v) {
          const auto lr = P::coef(cf, 2 * (D * cc + v)), li = P::coef(cf, 2 * (D * cc + v) + 1);
          yr = P::mac(yr, h[v].re, lr);
          yr = P::mac(yr, h[v].im, li);
          yi = P::mac(yi, h[v].im, lr);
          yi = P::mac(yi, P::neg(h[v].re), li);
        }
        yb[a * D + (cc ^ a)] = P::make(P::norm(yr), P::norm(yi));
      }
      __syncwarp(mask);
      Cx<P> y[D];
#pragma unroll
      for (int u = 0; u < D; ++u) {
        const E e = yb[u * D + (a ^ u)];
        y[u] = Cx<P>{P::re(e), P::im(e)};
      }
      __syncwarp(mask);
#pragma unroll
      for (int x = 0; x < D; ++x) {
        const auto l0r = P::coef(cf, 2 * D * x), l0i = P::coef(cf, 2 * D * x + 1);
        R zr = t == 0 ? P::mul(y[0].re, l0r) : P::mac(acc[x].re, y[0].re, l0r);
        R zi = t == 0 ? P::mul(y[0].im, l0r) : P::mac(acc[x].im, y[0].im, l0r);
        zr = P::mac(zr, P::neg(y[0].im), l0i);
        zi = P::mac(zi, y[0].re, l0i);
#pragma unroll
        for (int u = 1; u < D; ++u) {
          const auto lr = P::coef(cf, 2 * (D * x + u)), li = P::coef(cf, 2 * (D * x + u) + 1);
          zr = P::mac(zr, y[u].re, lr);
          zr = P::mac(zr, P::neg(y[u].im), li);
          zi = P::mac(zi, y[u].im, lr);
          zi = P::mac(zi, y[u].re, li);
        }
        acc[x] = Cx<P>{P::norm(zr), P::norm(zi)};
      }
    }
    // every lane of the block has read its row before any lane writes a column
    __syncwarp(mask);
    const bool dblk = s == sp;
#pragma unroll
    for (int x = 0; x < D; ++x)
      if (!dblk || x >= a) bwrite<P, SM>(st, ib | dep(x), jb | dep(a), I.m, acc[x]);
  }
}

// ------------------------------------------------------------------ projections
// H <- Pi_b H Pi_b * scale: elements whose row or column has bit q != b become 0.
template <class P, bool SM>
__device__ void apply_projection(const Ctx& c, typename P::Elem* st, int q, int b, double scale) {
  const BatchItem& I = *c.I;
  const auto f = dcoef<P>(scale);
  for (int64_t o = int64_t(c.g) * kBT + threadIdx.x; o < I.stored; o += int64_t(c.G) * kBT) {
    uint64_t i, j;
    decode(o, I.m, i, j);
    typename P::Elem e = Acc<P, SM>::ld(st, o, I.m);
    if (int((i >> q) & 1) != b || int((j >> q) & 1) != b) {
      e = Conv<P>::from(0.0, 0.0);
    } else if (scale != 1.0) {
      e = P::make(P::norm(P::mul(P::re(e), f)), P::norm(P::mul(P::im(e), f)));
    }
    Acc<P, SM>::st(st, o, I.m, e);
  }
}

// ------------------------------------------------------------------ one request
template <class P, bool SM>
__device__ void run_item(Ctx& c, typename P::Elem* st, typename P::Elem* ybuf, double* red, double* tot,
                         int* s_flag) {
  using E = typename P::Elem;
  const BatchItem& I = *c.I;
  const BatchDesc& d = *c.d;
  E* gst = reinterpret_cast<E*>(I.state);
  // the operator: built from the request's initial state, or staged from the array
  if (I.init == 1) init_pure<P, SM>(c, st);
  else if (I.init == 2) init_pauli_sum<P, SM>(c, st);
  else if (SM)
    for (int64_t o = threadIdx.x; o < I.stored; o += kBT) st[sm_off<P>(o, I.m)] = __ldcg(gst + o);
  if (!gang_sync(c, s_flag)) return;
  for (int k = I.op_begin; k < I.op_end; ++k) {
    const BatchOp op = d.ops[k];
    if (op.form == BF_PTM1) {
      apply_ptm1<P, SM>(c, st, op);
    } else if (op.form == BF_KRAUS2) {
      apply_kraus<P, SM, 2>(c, st, op, ybuf);
    } else if (op.form == BF_KRAUS3) {
      apply_kraus<P, SM, 3>(c, st, op, ybuf);
    } else {
      // Born probabilities in FP64 over the diagonal, then the projection
      const int q = op.q[0];
      double v[2] = {0.0, 0.0};
      const int64_t N = int64_t(1) << I.n;
      const int M = 1 << I.m;
      for (int64_t i = int64_t(c.g) * kBT + threadIdx.x; i < N; i += int64_t(c.G) * kBT) {
        const int64_t t = i >> I.m;
        const E e = Acc<P, SM>::ld(st, tile_base(t, t, I.m) + (i & (M - 1)) * (M + 1), I.m);
        if ((i >> q) & 1) v[1] += P::to_double(P::re(e));
        else v[0] += P::to_double(P::re(e));
      }
      if (!gang_sum<2>(c, v, red, tot, s_flag, 0)) return;
      int b = op.outcome;
      double scale = 1.0;
      if (op.form == BF_MEASURE) {
        const double p0 = tot[0], p1 = tot[1];
        b = op.u * (p0 + p1) < p0 ? 0 : 1;
        const double pb = b ? p1 : p0;
        if (!(pb > 1e-300)) {
          if (threadIdx.x == 0 && c.g == 0) atomicCAS(d.status + c.it, 0, ORKAN_EZEROPROB);
          return;   // every gang member reaches the same decision
        }
        scale = 1.0 / pb;
        if (threadIdx.x == 0 && c.g == 0) {
          d.outcomes[I.meas_base + op.meas] = b;
          d.probs[I.meas_base + op.meas] = pb / (p0 + p1);
        }
      }
      // every member has read the diagonal (gang_sum) before anyone projects
      apply_projection<P, SM>(c, st, q, b, scale);
    }
    if (!gang_sync(c, s_flag)) return;
  }
  // readouts: Pauli strings S = sum_i sign(i) h[i ^ x, i] (the host applies i^{nY})
  const uint64_t* pm = reinterpret_cast<const uint64_t*>(d.aux + I.pauli_off);
  const int64_t N = int64_t(1) << I.n;
  for (int p = 0; p < I.npauli; ++p) {
    const uint64_t x = pm[3 * p], z = pm[3 * p + 1], y = pm[3 * p + 2];
    double v[2] = {0.0, 0.0};
    for (int64_t i = int64_t(c.g) * kBT + threadIdx.x; i < N; i += int64_t(c.G) * kBT) {
      const Cx<P> e = bread<P, SM>(st, uint64_t(i) ^ x, uint64_t(i), I.m);
      const double er = P::to_double(e.re), ei = P::to_double(e.im);
      if ((__popcll(~uint64_t(i) & y) + __popcll(uint64_t(i) & z)) & 1) { v[0] -= er; v[1] -= ei; }
      else { v[0] += er; v[1] += ei; }
    }
    if (!gang_sum<2>(c, v, red, tot, s_flag, 2 * p)) return;
    if (threadIdx.x == 0 && c.g == 0) {
      d.results[I.res + 2 * p] = tot[0];
      d.results[I.res + 2 * p + 1] = tot[1];
    }
  }
  // <psi|H|psi> = sum_i H_ii |psi_i|^2 + 2 Re sum_{i > j} conj(psi_i) H_ij psi_j
  if (I.psi_off >= 0) {
    const double2* psi = reinterpret_cast<const double2*>(d.aux + I.psi_off);
    double v[1] = {0.0};
    for (int64_t o = int64_t(c.g) * kBT + threadIdx.x; o < I.stored; o += int64_t(c.G) * kBT) {
      uint64_t i, j;
      decode(o, I.m, i, j);
      if (i >= uint64_t(N) || j >= uint64_t(N) || i < j) continue;
      const E e = Acc<P, SM>::ld(st, o, I.m);
      const double hr = P::to_double(P::re(e)), hi = P::to_double(P::im(e));
      const double2 a = psi[i], b = psi[j];
      // conj(a) h b
      const double tr = a.x * b.x + a.y * b.y, ti = a.x * b.y - a.y * b.x;
      const double val = hr * tr - hi * ti;
      v[0] += i == j ? val : 2.0 * val;
    }
    if (!gang_sum<1>(c, v, red, tot, s_flag, 2 * I.npauli)) return;
    if (threadIdx.x == 0 && c.g == 0) d.results[I.res + 2 * I.npauli] = tot[0];
  }
  if (SM) {
    __syncthreads();
    for (int64_t o = threadIdx.x; o < I.stored; o += kBT) __stcg(gst + o, st[sm_off<P>(o, I.m)]);
  }
}

template <class P>
__global__ void __launch_bounds__(kBT) batch_kernel(const __grid_constant__ BatchDesc d) {
  using E = typename P::Elem;
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ __align__(16) E ybuf[kBT / 8 * 64];
  __shared__ double red[4 * kBW];
  __shared__ double tot[4];
  __shared__ int s_slot, s_flag;
  E* sst = reinterpret_cast<E*>(dyn);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_slot = atomicAdd(d.counter, 1);
    __syncthreads();
    const int slot = s_slot;
    if (slot >= d.nslots) return;
    const int it = d.slot_item[slot];
    const BatchItem& I = d.items[it];
    if (ld_acquire(d.status + it) != 0) continue;   // the request has failed: nothing left to do
    Ctx c{&d, &I, it, slot - I.first_slot, I.gang, 0};
    if (I.smem) run_item<P, true>(c, sst, ybuf, red, tot, &s_flag);
    else run_item<P, false>(c, reinterpret_cast<E*>(I.state), ybuf, red, tot, &s_flag);
  }
}

template <class P>
cudaError_t launch_batch_t(const BatchDesc& d, int grid, size_t smem, cudaStream_t s) {
  cudaError_t err = cudaFuncSetAttribute(batch_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (err != cudaSuccess) return err;
  batch_kernel<P><<<grid, kBT, smem, s>>>(d);
  return cudaGetLastError();
}

template <class P>
cudaError_t occupancy_t(size_t smem, int* per_sm) {
  cudaError_t err = cudaFuncSetAttribute(batch_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_kernel<P>, kBT, smem);
}

}  // namespace

cudaError_t batch_occupancy(int dtype, size_t smem, int* per_sm) {
  switch (dtype) {
    case DT_C128: return occupancy_t<PolF64>(smem, per_sm);
    case DT_C64: return occupancy_t<PolF32>(smem, per_sm);
    default: return occupancy_t<PolDF64>(smem, per_sm);
  }
}

cudaError_t launch_batch(int dtype, const BatchDesc& d, int grid, size_t smem, cudaStream_t stream) {
  if (grid <= 0 || d.nslots <= 0) return cudaSuccess;
  switch (dtype) {
    case DT_C128: return launch_batch_t<PolF64>(d, grid, smem, stream);
    case DT_C64: return launch_batch_t<PolF32>(d, grid, smem, stream);
    default: return launch_batch_t<PolDF64>(d, grid, smem, stream);
  }
}

}  // namespace orkan
