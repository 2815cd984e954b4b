// Host side of the Orkan GB300 library: the C ABI of include/orkan.h, the
// FP64 preparation of every op (Pauli transfer matrices, Sec. II-A Eq. 3),
// and the planner that fuses consecutive ops into passes.
//
// An op on qubits A is classified by its high qubits A>=m (Sec. III-C: the
// number of tiles a k-local update spans grows as 2^(2 |A>=m|)).  Consecutive
// ops are fused while the union of their high qubits has at most two
// elements and the tile group still fits the shared-memory budget; a pass is
// then one read and one write of the tiled array.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <tuple>
#include <complex>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/orkan.h"
#include "orkan_internal.h"

using cd = std::complex<double>;
using namespace orkan;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* where) {
  return fail(ORKAN_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define ORKAN_CUDA(call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
  } while (0)

int elem_size(int dtype) { return dtype == DT_C64 ? 8 : 16; }
bool valid_dtype(int dtype) { return dtype == DT_C128 || dtype == DT_C64 || dtype == DT_DF64; }

// ------------------------------------------------------------------ Pauli algebra (FP64)
const cd kPauli[4][4] = {
    {1, 0, 0, 1},                                  // I
    {0, 1, 1, 0},                                  // X
    {0, cd(0, -1), cd(0, 1), 0},                   // Y
    {1, 0, 0, -1},                                 // Z
};

// d x d complex matrices, row-major.
using Mat = std::vector<cd>;

Mat matmul(const Mat& A, const Mat& B, int d) {
  Mat C(d * d, 0.0);
  for (int i = 0; i < d; ++i)
    for (int k = 0; k < d; ++k) {
      const cd a = A[i * d + k];
      if (a == 0.0) continue;
      for (int j = 0; j < d; ++j) C[i * d + j] += a * B[k * d + j];
    }
  return C;
}
Mat dagger(const Mat& A, int d) {
  Mat B(d * d);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) B[j * d + i] = std::conj(A[i * d + j]);
  return B;
}
Mat pauli_string(int a, int k) {
  // P_a = sigma_{a_{k-1}} (x) ... (x) sigma_{a_0}
  Mat P{1.0};
  int dim = 1;
  for (int l = k - 1; l >= 0; --l) {
    const int s = (a >> (2 * l)) & 3;
    Mat Q(dim * 2 * dim * 2);
    for (int i = 0; i < dim; ++i)
      for (int j = 0; j < dim; ++j)
        for (int x = 0; x < 2; ++x)
          for (int y = 0; y < 2; ++y)
            Q[(2 * i + x) * (2 * dim) + (2 * j + y)] = P[i * dim + j] * kPauli[s][2 * x + y];
    P.swap(Q);
    dim *= 2;
  }
  return P;
}

// k = 1 on fixed-size arrays (no heap traffic per product): every op of a
// circuit goes through here once, so its host cost bounds small-operator rates.
std::vector<double> ptm1(const std::vector<Mat>& kraus, bool adjoint) {
  std::vector<double> R(16, 0.0);
  for (int b = 0; b < 4; ++b) {
    cd img[4] = {0.0, 0.0, 0.0, 0.0};   // Phi(P_b) (or Phi*(P_b)), row-major 2 x 2
    for (const Mat& K : kraus) {
      // M = adjoint ? K^dagger : K; img += M P_b M^dagger
      cd M[4];
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) M[2 * i + j] = adjoint ? std::conj(K[2 * j + i]) : K[2 * i + j];
      cd MP[4];
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) MP[2 * i + j] = M[2 * i] * kPauli[b][j] + M[2 * i + 1] * kPauli[b][2 + j];
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) img[2 * i + j] += MP[2 * i] * std::conj(M[2 * j]) + MP[2 * i + 1] * std::conj(M[2 * j + 1]);
    }
    for (int a = 0; a < 4; ++a) {
      // tr(P_a img) / 2
      const cd tr = kPauli[a][0] * img[0] + kPauli[a][1] * img[2] + kPauli[a][2] * img[1] + kPauli[a][3] * img[3];
      R[4 * a + b] = 0.5 * tr.real();
    }
  }
  return R;
}

// Pauli transfer matrix R[a][b] = 2^-k Re tr(P_a Phi(P_b)) of the Kraus set.
std::vector<double> ptm(int k, const std::vector<Mat>& kraus, bool adjoint) {
  if (k == 1) return ptm1(kraus, adjoint);
  const int d = 1 << k, np = 1 << (2 * k);
  std::vector<Mat> P(np);
  for (int a = 0; a < np; ++a) P[a] = pauli_string(a, k);
  std::vector<double> R(np * np, 0.0);
  for (int b = 0; b < np; ++b) {
    Mat img(d * d, 0.0);
    for (const Mat& K : kraus) {
      const Mat Kd = dagger(K, d);
      const Mat t = adjoint ? matmul(matmul(Kd, P[b], d), K, d) : matmul(matmul(K, P[b], d), Kd, d);
      for (int i = 0; i < d * d; ++i) img[i] += t[i];
    }
    for (int a = 0; a < np; ++a) {
      const Mat pa = matmul(P[a], img, d);
      cd tr = 0.0;
      for (int i = 0; i < d; ++i) tr += pa[i * d + i];
      R[a * np + b] = tr.real() / d;
    }
  }
  return R;
}

Mat read_mat(const double* p, int d) {
  Mat A(d * d);
  for (int i = 0; i < d * d; ++i) A[i] = cd(p[2 * i], p[2 * i + 1]);
  return A;
}
// Re-express a two-qubit matrix given on (q0, q1) with q0 > q1 in the ascending order.
Mat swap_local_bits(const Mat& A) {
  auto p = [](int i) { return ((i & 1) << 1) | (i >> 1); };
  Mat B(16);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) B[p(i) * 4 + p(j)] = A[i * 4 + j];
  return B;
}

// ------------------------------------------------------------------ planned ops
struct HostOp {
  int kind = OP_PTM1;
  int nq = 1;
  int q[3] = {0, 0, 0};        // ascending
  std::vector<double> R;       // single-qubit ops: full 4x4 PTM (for composition)
  std::vector<double> coef;    // kind-specific FP64 coefficients (2- and 3-qubit ops)
  std::vector<long long> codes;  // monomial ops: permutation and phase codes
  // single-Kraus ops (k <= 2): the map is L (.) L^dagger with L on q[] (bit l of
  // L's index on q[l]), the adjoint already applied on observables; consecutive
  // in-tile ones compose into one block for the tensor-core pass
  Mat L;
  bool has_L = false;
};

// A unitary is monomial with quarter-turn phases when every row holds exactly
// one non-zero entry, equal to one of 1, i, -1, -i (tested exactly).  Then
// V[i][p_i] = i^{q_i}; returns false otherwise.
bool monomial(const Mat& V, int d, std::vector<long long>* p, std::vector<long long>* q) {
  p->assign(d, 0);
  q->assign(d, 0);
  std::vector<int> used(d, 0);
  for (int i = 0; i < d; ++i) {
    int nz = 0;
    for (int j = 0; j < d; ++j) {
      const cd v = V[i * d + j];
      if (v == cd(0.0, 0.0)) continue;
      ++nz;
      int code;
      if (v == cd(1, 0)) code = 0;
      else if (v == cd(0, 1)) code = 1;
      else if (v == cd(-1, 0)) code = 2;
      else if (v == cd(0, -1)) code = 3;
      else return false;
      (*p)[i] = j;
      (*q)[i] = code;
    }
    if (nz != 1 || used[(*p)[i]]) return false;
    used[(*p)[i]] = 1;
  }
  return true;
}

std::vector<double> mat4mul(const std::vector<double>& A, const std::vector<double>& B) {
  std::vector<double> C(16, 0.0);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += A[i * 4 + k] * B[k * 4 + j];
      C[i * 4 + j] = s;
    }
  return C;
}

// Coefficients of a single-qubit op from its transfer matrix R.
std::vector<double> coef_1q(int kind, const std::vector<double>& R) {
  std::vector<double> c;
  if (kind == OP_PTM1_U) {
    for (int i = 1; i < 4; ++i)
      for (int j = 1; j < 4; ++j) c.push_back(0.5 * R[i * 4 + j]);
  } else if (kind == OP_PTM1_AD) {
    const double R00 = R[0], R03 = R[3], R30 = R[12], R33 = R[15];
    c = {0.5 * (R00 + R30 + R03 + R33), 0.5 * (R00 + R30 - R03 - R33), 0.5 * (R00 - R30 + R03 - R33),
         0.5 * (R00 - R30 - R03 + R33), R[5], R[9]};
  } else {
    for (int i = 0; i < 16; ++i) c.push_back(0.5 * R[i]);
  }
  return c;
}

bool is_ad_pattern(const std::vector<double>& R) {
  const int zeros[] = {1, 2, 4, 7, 8, 11, 13, 14};
  for (int z : zeros)
    if (R[z] != 0.0) return false;
  return R[5] == R[10] && R[6] == -R[9];
}
bool is_unitary_pattern(const std::vector<double>& R) {
  return R[0] == 1.0 && R[1] == 0.0 && R[2] == 0.0 && R[3] == 0.0 && R[4] == 0.0 && R[8] == 0.0 && R[12] == 0.0;
}

}  // namespace

// ------------------------------------------------------------------ the handle
struct orkan_ctx {
  Geometry g{};
  int dtype = DT_C128;
  int picture = ORKAN_STATE;
  int device = 0;
  size_t bytes = 0;
  void* d_state = nullptr;
  bool external = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int fusion = 8;
  bool compose = true;
  std::vector<HostOp> pending;
  // single-Kraus single-qubit ops held back, at most one per physical qubit:
  // the next op on that qubit either absorbs it (a two-qubit single-Kraus op)
  // or is preceded by it; every flush releases them
  std::vector<HostOp> held;
  double* d_partials = nullptr;
  double* d_res = nullptr;
  double* h_res = nullptr;   // pinned
  void* d_upload = nullptr;  // grow-only staging buffer for init uploads (no per-call cudaMalloc/cudaFree,
  size_t upload_cap = 0;     // which could synchronise the device under concurrent requests)
  int64_t n_passes = 0, n_ops = 0, n_launches = 0;
  bool timing = false;
  bool capturing = false;
  double work_ops = 0.0, work_bytes = 0.0;   // algorithmic ALU ops / bytes of the timed passes
  int phys[64];            // qubit relabelling: logical qubit -> physical bit position
  int cap_phys[64];        // the map when the running graph capture began
  int auto_relabel = 0;    // 1: orkan_run_circuit moves a circuit's most used qubits into the tile
  int tc_mode = 0;              // tensor-core pass for composed in-tile runs: 0 off, 1 auto, 2 always
  int32_t* d_err = nullptr;     // device error word of the tensor-core pass (allocated on first use)
  std::vector<cudaEvent_t> ev_free;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_used;
};

namespace {

// Algorithmic arithmetic per element of each op form: pipe instructions of the
// formula as written (double-float: add 11, mul 4, multiply-add 12,
// renormalise 3, halve 2 FP32 ops; FP64 / FP32: one op each), excluding
// addressing and data movement.  Used for the ALU roofline of timed passes.
double alu_ops_per_elem(int dtype, int kind) {
  const bool dfl = dtype == DT_DF64;
  switch (kind) {
    case OP_PTM1_U: return dfl ? 366.0 / 4 : 36.0 / 4;
    case OP_PTM1: return dfl ? 520.0 / 4 : 48.0 / 4;
    case OP_PTM1_AD: return dfl ? 152.0 / 4 : 16.0 / 4;
    case OP_U2: return dfl ? 364.0 : 32.0;
    case OP_PTM2: return dfl ? 7392.0 / 16 : 640.0 / 16;
    case OP_K3: return dfl ? 748.0 : 64.0;   // per Kraus term: row and column sweeps, 8 complex MACs each
    default: return 0.0;   // monomial ops: no arithmetic
  }
}

int rows_log2_for(const orkan_ctx* h, int nh) {
  // 2^(2 nh) tiles x 2^rl rows x M columns within a 64 KiB shared-memory budget
  const int64_t budget = 64 * 1024;
  const int64_t per_row = (int64_t(1) << (2 * nh)) * (int64_t(1) << h->g.m) * elem_size(h->dtype);
  int rl = 0;
  while (rl < h->g.m && (per_row << (rl + 1)) <= budget) ++rl;
  return rl;
}

struct PassShape {
  int nh = 0;
  int high[2] = {0, 0};
  int max_low = -1;
};

PassShape shape_of(const orkan_ctx* h, const std::vector<HostOp>& ops, const HostOp* extra) {
  PassShape s;
  std::vector<int> high;
  auto add = [&](const HostOp& op) {
    for (int l = 0; l < op.nq; ++l) {
      const int q = op.q[l];
      if (q >= h->g.m) {
        if (std::find(high.begin(), high.end(), q) == high.end()) high.push_back(q);
      } else {
        s.max_low = std::max(s.max_low, q);
      }
    }
  };
  for (const auto& op : ops) add(op);
  if (extra) add(*extra);
  std::sort(high.begin(), high.end());
  s.nh = int(high.size());
  for (int i = 0; i < s.nh && i < 2; ++i) s.high[i] = high[i];
  return s;
}

int slots_upper_bound(const orkan_ctx* h, const HostOp& op) {
  const bool paired = h->dtype == DT_DF64;
  return op.nq == 1 ? coef_slots(OP_PTM1, paired) : coef_slots(op.kind, paired);
}

bool tc_run(const orkan_ctx* h);
bool tc_op_ok(const orkan_ctx* h, const HostOp& op);

bool fits(const orkan_ctx* h, const HostOp& op) {
  if (h->pending.empty()) return true;
  if (tc_run(h) && tc_op_ok(h, op)) return true;   // the run stays one composed block
  if (int(h->pending.size()) >= std::min(h->fusion, kMaxOps)) return false;
  const PassShape s = shape_of(h, h->pending, &op);
  if (s.nh > 2) return false;
  if (s.max_low >= rows_log2_for(h, s.nh)) return false;
  int slots = slots_upper_bound(h, op);
  for (const auto& p : h->pending) slots += slots_upper_bound(h, p);
  return slots <= kMaxCoef;
}

// One FP64 coefficient into an 8-byte slot in the policy's format: C128 the
// double, C64 the float (low half), DF64 the (hi, lo) float pair.
void pack_slot(int dtype, double* slot, double v) {
  if (dtype == DT_C128) {
    *slot = v;
  } else if (dtype == DT_C64) {
    const float pair[2] = {(float)v, 0.0f};
    std::memcpy(slot, pair, 8);
  } else {
    const float hi = (float)v;
    const float pair[2] = {hi, (float)(v - (double)hi)};
    std::memcpy(slot, pair, 8);
  }
}

// The coefficients c of one op (kind-specific FP64 list) into slots, in the
// layout its kernel body reads; returns the slots written.  DF64 forms with a
// paired body (PTM1, PTM1_U, PTM1_AD) take each coefficient use as a lane
// pair of double-float values, the hi pair then the lo pair: (v, v) for a real
// factor, (-v, v) where the body multiplies the lane swap (x.im, x.re), i.e.
// i x, and (v, -v) for -i x.  The other forms and dtypes: one slot each.
int pack_op_coefs(int dtype, int kind, const std::vector<double>& c, double* slots) {
  const bool paired = dtype == DT_DF64 && (kind == OP_PTM1 || kind == OP_PTM1_U || kind == OP_PTM1_AD);
  if (!paired) {
    for (size_t i = 0; i < c.size(); ++i) pack_slot(dtype, &slots[i], c[i]);
    return int(c.size());
  }
  int k = 0;
  auto pair = [&](double v0, double v1) {
    const float h0 = (float)v0, h1 = (float)v1;
    const float hi[2] = {h0, h1}, lo[2] = {(float)(v0 - (double)h0), (float)(v1 - (double)h1)};
    std::memcpy(&slots[2 * k], hi, 8);
    std::memcpy(&slots[2 * k + 1], lo, 8);
    ++k;
  };
  if (kind == OP_PTM1) {            // 4 x 4, column 2 multiplies i (b - c)
    for (int i = 0; i < 16; ++i) {
      if (i % 4 == 2) pair(-c[i], c[i]);
      else pair(c[i], c[i]);
    }
  } else if (kind == OP_PTM1_U) {   // 3 x 3, column 1 multiplies i (b - c)
    for (int i = 0; i < 9; ++i) {
      if (i % 3 == 1) pair(-c[i], c[i]);
      else pair(c[i], c[i]);
    }
  } else {                          // PTM1_AD: al, be, ga, de, rho; sig for h10 (+i), for h01 (-i)
    for (int i = 0; i < 5; ++i) pair(c[i], c[i]);
    pair(-c[5], c[5]);
    pair(c[5], -c[5]);
  }
  return 2 * k;
}

// Event pair bracketing one timed pass (pooled events); none while capturing.
int timing_begin(orkan_ctx* h, std::pair<cudaEvent_t, cudaEvent_t>* ev) {
  *ev = {nullptr, nullptr};
  if (!h->timing || h->capturing) return ORKAN_OK;
  for (int i = 0; i < 2; ++i) {
    cudaEvent_t e;
    if (!h->ev_free.empty()) {
      e = h->ev_free.back();
      h->ev_free.pop_back();
    } else {
      ORKAN_CUDA(cudaEventCreate(&e));
    }
    (i == 0 ? ev->first : ev->second) = e;
  }
  ORKAN_CUDA(cudaEventRecord(ev->first, h->stream));
  return ORKAN_OK;
}
int timing_end(orkan_ctx* h, const std::pair<cudaEvent_t, cudaEvent_t>& ev, double alu_ops) {
  if (!ev.first) return ORKAN_OK;
  ORKAN_CUDA(cudaEventRecord(ev.second, h->stream));
  h->ev_used.push_back(ev);
  h->work_ops += alu_ops;
  h->work_bytes += 2.0 * double(h->bytes);
  return ORKAN_OK;
}

// A three-qubit op: its own launch, after the pending fused ops.
int run_k3(orkan_ctx* h, const HostOp& op) {
  K3Desc d;
  std::memset(&d, 0, sizeof(d));
  const int64_t S = int64_t(1) << (h->g.n - 3);
  d.nblocks = S * (S + 1) / 2;
  d.m = h->g.m;
  for (int l = 0; l < 3; ++l) d.q[l] = op.q[l];
  if (op.kind == OP_MONO3) {
    d.form = 1;
    for (int i = 0; i < 16; ++i) std::memcpy(&d.coef[i], &op.codes[i], 8);
  } else {
    d.form = 0;
    d.r = int(op.coef.size() / 128);
    for (size_t i = 0; i < op.coef.size(); ++i) pack_slot(h->dtype, &d.coef[i], op.coef[i]);
  }
  std::pair<cudaEvent_t, cudaEvent_t> ev;
  if (int st = timing_begin(h, &ev)) return st;
  ORKAN_CUDA(launch_k3(h->dtype, h->d_state, d, h->stream));
  const double elems = double(h->g.ntiles) * double(int64_t(1) << (2 * h->g.m));
  if (int st = timing_end(h, ev, elems * alu_ops_per_elem(h->dtype, op.kind) * std::max(d.r, 1))) return st;
  h->n_passes += 1;
  h->n_ops += 1;
  h->n_launches += 1;
  return ORKAN_OK;
}

// ------------------------------------------------------------------ tensor-core pass
constexpr int kTcMaxOps = 64;

bool tc_op_ok(const orkan_ctx* h, const HostOp& op) {
  if (!op.has_L || op.nq > 3) return false;
  for (int l = 0; l < op.nq; ++l)
    if (op.q[l] >= h->g.m) return false;
  return true;
}
// The pending run may become one tensor-core pass (every op in-tile with a single Kraus operator).
bool tc_run(const orkan_ctx* h) {
  // fusion depth 1 keeps the plain one-pass-per-op path
  if (h->tc_mode == 0 || h->fusion < 2 || h->dtype != DT_C64 || h->g.m != 5 || h->pending.empty()) return false;
  for (const HostOp& op : h->pending)
    if (!tc_op_ok(h, op)) return false;
  return true;
}
// ... and is worth it: mode 2 always; mode 1 with two dense two-qubit ops or six ops.
bool tc_take(const orkan_ctx* h) {
  if (!tc_run(h)) return false;
  if (h->tc_mode == 2) return true;
  int dense2 = 0;
  for (const HostOp& op : h->pending) {
    if (op.nq == 3) return true;   // a three-qubit op joins a run only as part of a tensor-core pass
    dense2 += op.nq == 2 && op.codes.empty();
  }
  return dense2 >= 2 || h->pending.size() >= 6;
}
// The pending run can only leave as a tensor-core pass: it is longer than a
// fused pass holds or holds a three-qubit op.
bool tc_required(const orkan_ctx* h) {
  if (int(h->pending.size()) > kMaxOps) return true;
  for (const HostOp& op : h->pending)
    if (op.nq == 3) return true;
  return false;
}

// L_blk = L_k ... L_1 over the run, each L embedded on the tile's m qubits (FP64).
int flush_tc(orkan_ctx* h) {
  const int M = 1 << h->g.m;
  Mat blk(M * M, 0.0);
  for (int i = 0; i < M; ++i) blk[i * M + i] = 1.0;
  for (const HostOp& op : h->pending) {
    const int d = 1 << op.nq;
    int mask = 0;
    for (int l = 0; l < op.nq; ++l) mask |= 1 << op.q[l];
    auto loc = [&](int r) {
      int a = 0;
      for (int l = 0; l < op.nq; ++l) a |= ((r >> op.q[l]) & 1) << l;
      return a;
    };
    Mat E(M * M, 0.0);
    for (int r = 0; r < M; ++r)
      for (int c = 0; c < M; ++c)
        if ((r & ~mask) == (c & ~mask)) E[r * M + c] = op.L[loc(r) * d + loc(c)];
    blk = matmul(E, blk, M);
  }
  TcDesc d;
  d.ntiles = h->g.ntiles;
  d.err = h->d_err;
  for (int i = 0; i < M * M; ++i) d.u[i] = make_float2(float(blk[i].real()), float(blk[i].imag()));
  const int64_t nops = int64_t(h->pending.size());
  h->pending.clear();
  std::pair<cudaEvent_t, cudaEvent_t> ev;
  if (int st = timing_begin(h, &ev)) return st;
  ORKAN_CUDA(launch_tc(h->d_state, d, h->stream));
  if (int st = timing_end(h, ev, 0.0)) return st;
  h->n_passes += 1;
  h->n_ops += nops;
  h->n_launches += 1;
  return ORKAN_OK;
}

int flush_pass(orkan_ctx* h) {
  if (h->pending.empty()) return ORKAN_OK;
  if (tc_take(h)) return flush_tc(h);
  if (tc_required(h)) {   // the planner never builds such a run; refuse rather than overrun the pass descriptor
    h->pending.clear();
    return fail(ORKAN_EINVAL, "internal: a run of more than 16 ops or with a three-qubit op is not a tensor-core run");
  }
  const PassShape s = shape_of(h, h->pending, nullptr);
  // in-tile passes run with four independent tiles per work item, on the
  // one-high-qubit group geometry
  const int rl = rows_log2_for(h, s.nh == 0 ? 1 : s.nh);
  PassDesc d;
  std::memset(&d, 0, sizeof(d));
  d.m = h->g.m;
  d.h = s.nh;
  for (int i = 0; i < s.nh; ++i) d.hpos[i] = s.high[i] - h->g.m;
  d.rows_log2 = rl;
  d.chunks_log2 = h->g.m - rl;
  d.nt_c = h->g.Nt >> s.nh;
  // A chunked pass splits tile rows over work items; in a diagonal group the
  // mirrored slots would then read rows another item is writing, so those
  // groups go to the full-height diagonal kernel instead.
  d.skip_diag = d.chunks_log2 > 0 ? 1 : 0;
  const int64_t groups = d.skip_diag ? d.nt_c * (d.nt_c - 1) / 2 : d.nt_c * (d.nt_c + 1) / 2;
  d.n_items = groups << d.chunks_log2;
  d.n_tiles = h->g.ntiles;
  if (s.nh == 0) d.n_items = (h->g.ntiles + 3) / 4;
  int slot = 0;
  double work_per_elem = 0.0;   // algorithmic ALU operations per element of the pass
  for (const HostOp& op : h->pending) {
    work_per_elem += alu_ops_per_elem(h->dtype, op.nq == 1 && !op.codes.empty() ? OP_MONO1 : op.kind);
    // native FP64 applies an AD-form map with a real off-diagonal factor in 12 operations per block
    if (h->dtype == DT_C128 && op.kind == OP_PTM1_AD && op.codes.empty() && op.R[9] == 0.0) work_per_elem -= 1.0;
    PassOp& po = d.ops[d.nops++];
    po.kind = op.kind;
    po.nq = op.nq;
    for (int l = 0; l < op.nq; ++l) {
      const int q = op.q[l];
      if (q < h->g.m) {
        po.rbit[l] = q;
        po.cbit[l] = q;
      } else {
        const int p = (q == s.high[0]) ? 0 : 1;
        po.rbit[l] = rl + p;
        po.cbit[l] = h->g.m + p;
      }
    }
    po.coef = slot;
    if (op.kind == OP_PTM2) d.has_ptm2 = 1;
    if (op.nq == 1 && !op.codes.empty()) {
      po.kind = OP_MONO1;
      for (long long v : op.codes) std::memcpy(&d.coef[slot++], &v, 8);
      continue;
    }
    const std::vector<double> c = op.nq == 1 ? coef_1q(op.kind, op.R) : op.coef;
    slot += pack_op_coefs(h->dtype, op.kind, c, &d.coef[slot]);
    for (long long v : op.codes) std::memcpy(&d.coef[slot++], &v, 8);
  }
  const int64_t nops = int64_t(h->pending.size());
  h->pending.clear();
  std::pair<cudaEvent_t, cudaEvent_t> ev;
  if (int st = timing_begin(h, &ev)) return st;
  int nlaunch = 0;
  ORKAN_CUDA(launch_pass(h->dtype, h->d_state, d, h->stream, &nlaunch));
  double alu = 0.0;
  const double elems = double(h->g.ntiles) * double(int64_t(1) << (2 * h->g.m));
  alu = elems * work_per_elem;
  if (int st = timing_end(h, ev, alu)) return st;
  h->n_passes += 1;
  h->n_ops += nops;
  h->n_launches += nlaunch;
  return ORKAN_OK;
}

bool tc_run(const orkan_ctx* h);
bool tc_op_ok(const orkan_ctx* h, const HostOp& op);
bool tc_required(const orkan_ctx* h);

int enqueue_now(orkan_ctx* h, HostOp op) {
  if (op.nq == 3) {
    // an in-tile three-qubit single-Kraus op joins a tensor-core run (complex64, m = 5)
    const bool joins = h->tc_mode != 0 && h->fusion >= 2 && h->dtype == DT_C64 && h->g.m == 5 &&
                       tc_op_ok(h, op) && (h->pending.empty() || tc_run(h));
    if (!joins) {
      if (int st = flush_pass(h)) return st;
      return run_k3(h, op);
    }
    h->pending.push_back(std::move(op));
    if (int(h->pending.size()) >= kTcMaxOps) return flush_pass(h);
    return ORKAN_OK;
  }
  // a run that can only leave as a tensor-core pass (longer than a fused pass
  // holds, or holding a three-qubit op) ends before an op that cannot join
  // it -- before composition too, which would otherwise merge such an op into
  // the run's last op and turn the run into an ordinary pass it cannot be
  if (!h->pending.empty() && tc_required(h) && !tc_op_ok(h, op))
    if (int st = flush_pass(h)) return st;
  // compose consecutive single-qubit ops on the same qubit (FP64, on the host)
  if (h->compose && op.nq == 1 && !h->pending.empty()) {
    HostOp& last = h->pending.back();
    if (last.nq == 1 && last.q[0] == op.q[0]) {
      last.R = mat4mul(op.R, last.R);
      if (last.has_L && op.has_L) last.L = matmul(op.L, last.L, 2);
      else last.has_L = false;
      last.codes.clear();
      if (!(last.kind == op.kind && (op.kind == OP_PTM1_U || op.kind == OP_PTM1_AD))) {
        last.kind = is_unitary_pattern(last.R) ? OP_PTM1_U : (is_ad_pattern(last.R) ? OP_PTM1_AD : OP_PTM1);
      }
      h->n_ops += 1;
      return ORKAN_OK;
    }
  }
  if (!fits(h, op)) {
    const int st = flush_pass(h);
    if (st != ORKAN_OK) return st;
  }
  h->pending.push_back(std::move(op));
  const int limit = tc_run(h) ? kTcMaxOps : std::min(h->fusion, kMaxOps);
  if (int(h->pending.size()) >= limit) return flush_pass(h);
  return ORKAN_OK;
}

// Release the held single-qubit ops (they commute: distinct qubits), in qubit order.
int release_held(orkan_ctx* h) {
  std::vector<HostOp> held;
  held.swap(h->held);
  std::sort(held.begin(), held.end(), [](const HostOp& a, const HostOp& b) { return a.q[0] < b.q[0]; });
  for (HostOp& op : held) {
    h->n_ops -= 1;   // counted when it was held
    if (int st = enqueue_now(h, std::move(op))) return st;
  }
  return ORKAN_OK;
}

// Every op goes through here.  With fusion and composition on, a
// single-Kraus single-qubit op is held back; a later single-qubit op on the
// same qubit composes with it, a single-Kraus two-qubit op on it absorbs it
// (L2 (L1 (x) I), one 4 x 4 product in FP64: the held op moves forward past
// ops on other qubits only, with which it commutes), and any other op on it
// releases it first.  Noisy layered circuits (a single-qubit gate on every
// qubit, then two-qubit gates on pairs) thus run their single-qubit gates
// inside the two-qubit ones.
int enqueue(orkan_ctx* h, HostOp op) {
  const bool fold = h->compose && h->fusion >= 2;
  if (!fold) return enqueue_now(h, std::move(op));
  if (op.nq == 1 && op.has_L) {
    for (HostOp& held : h->held)
      if (held.q[0] == op.q[0]) {
        held.R = mat4mul(op.R, held.R);
        held.L = matmul(op.L, held.L, 2);
        held.codes.clear();
        held.kind = is_unitary_pattern(held.R) ? OP_PTM1_U : (is_ad_pattern(held.R) ? OP_PTM1_AD : OP_PTM1);
        h->n_ops += 1;
        return ORKAN_OK;
      }
    h->held.push_back(std::move(op));
    h->n_ops += 1;
    return ORKAN_OK;
  }
  if (op.nq == 2 && op.has_L && op.kind == OP_U2) {   // a permutation gate stays a permutation
    bool folded = false;
    for (int l = 0; l < 2; ++l)
      for (size_t i = 0; i < h->held.size(); ++i)
        if (h->held[i].q[0] == op.q[l]) {
          // L <- L (u on local bit l)
          const Mat& u = h->held[i].L;
          Mat E(16, 0.0);
          for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
              if (((a ^ b) & ~(1 << l)) == 0) E[a * 4 + b] = u[((a >> l) & 1) * 2 + ((b >> l) & 1)];
          op.L = matmul(op.L, E, 4);
          h->held.erase(h->held.begin() + long(i));
          folded = true;
          break;
        }
    if (folded) {
      op.coef.resize(32);
      for (int i = 0; i < 16; ++i) {
        op.coef[2 * i] = op.L[i].real();
        op.coef[2 * i + 1] = op.L[i].imag();
      }
    }
    return enqueue_now(h, std::move(op));
  }
  // any other op releases the held ops on its qubits first (a three-qubit op all of them)
  if (op.nq == 3) {
    if (int st = release_held(h)) return st;
    return enqueue_now(h, std::move(op));
  }
  for (size_t i = 0; i < h->held.size();) {
    bool touches = false;
    for (int l = 0; l < op.nq; ++l) touches |= h->held[i].q[0] == op.q[l];
    if (touches) {
      HostOp held = std::move(h->held[i]);
      h->held.erase(h->held.begin() + long(i));
      h->n_ops -= 1;
      if (int st = enqueue_now(h, std::move(held))) return st;
    } else {
      ++i;
    }
  }
  return enqueue_now(h, std::move(op));
}

// Everything issued so far goes to the stream: held ops, then the pending pass.
int flush_pending(orkan_ctx* h) {
  if (!h->held.empty())
    if (int st = release_held(h)) return st;
  return flush_pass(h);
}

int check_handle(orkan_h h) {
  if (!h) return fail(ORKAN_EINVAL, "null handle");
  return ORKAN_OK;
}
// Calls that wait for the device or read results cannot be recorded into a graph.
int check_blocking(orkan_h h) {
  if (int st = check_handle(h)) return st;
  if (h->capturing) return fail(ORKAN_EINVAL, "not allowed while capturing a graph (blocking call)");
  return ORKAN_OK;
}

int check_qubits_n(int n, int k, const int* qubits) {
  if (k < 1 || k > 3 || !qubits) return fail(ORKAN_EINVAL, "k must be 1, 2 or 3 with a qubit list");
  for (int l = 0; l < k; ++l)
    if (qubits[l] < 0 || qubits[l] >= n) return fail(ORKAN_EINVAL, "qubit out of range");
  for (int l = 0; l < k; ++l)
    for (int l2 = l + 1; l2 < k; ++l2)
      if (qubits[l] == qubits[l2]) return fail(ORKAN_EINVAL, "repeated qubit");
  return ORKAN_OK;
}
int check_qubits(const orkan_ctx* h, int k, const int* qubits) { return check_qubits_n(h->g.n, k, qubits); }

// ------------------------------------------------------------------ qubit relabelling
void reset_labels(orkan_ctx* h) {
  for (int q = 0; q < 64; ++q) h->phys[q] = q;
}
bool labels_identity(const orkan_ctx* h) {
  for (int q = 0; q < h->g.n; ++q)
    if (h->phys[q] != q) return false;
  return true;
}
// physical index of logical basis index l: bit q of l moves to bit phys[q]
uint64_t phys_index(const orkan_ctx* h, uint64_t l) {
  uint64_t p = 0;
  for (int q = 0; q < h->g.n; ++q) p |= ((l >> q) & 1u) << h->phys[q];
  return p;
}
void map_qubits(const orkan_ctx* h, int k, const int* q, int* out) {
  for (int l = 0; l < k; ++l) out[l] = h->phys[q[l]];
}

// Build the planned op for a k-local Kraus set given in the caller's qubit order.
// adj: build the adjoint map (observable handles).
int make_op_adj(bool adj, int k, const int* qubits, const std::vector<Mat>& kraus_in, bool unitary, HostOp* out) {
  HostOp op;
  op.nq = k;
  std::vector<Mat> kraus = kraus_in;
  if (k == 3) {
    // caller bit l <-> qubits[l]; re-index to ascending qubit order
    int order[3] = {0, 1, 2};
    std::sort(order, order + 3, [&](int x, int y) { return qubits[x] < qubits[y]; });
    int rank[3];
    for (int l = 0; l < 3; ++l) {
      op.q[l] = qubits[order[l]];
      rank[order[l]] = l;
    }
    auto perm = [&](int x) { return ((x & 1) << rank[0]) | (((x >> 1) & 1) << rank[1]) | (((x >> 2) & 1) << rank[2]); };
    for (auto& K : kraus) {
      Mat B(64);
      for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) B[perm(i) * 8 + perm(j)] = K[i * 8 + j];
      // the adjoint map applies L^dagger (.) L = M (.) M^dagger with M = L^dagger
      K = adj ? dagger(B, 8) : B;
    }
    if (kraus.size() == 1) {
      op.L = kraus[0];
      op.has_L = true;
    }
    std::vector<long long> pp, qq;
    if (unitary && monomial(kraus[0], 8, &pp, &qq)) {
      op.kind = OP_MONO3;
      op.codes = pp;
      op.codes.insert(op.codes.end(), qq.begin(), qq.end());
    } else {
      op.kind = OP_K3;
      op.coef.resize(128 * kraus.size());
      for (size_t t = 0; t < kraus.size(); ++t)
        for (int i = 0; i < 64; ++i) {
          op.coef[128 * t + 2 * i] = kraus[t][i].real();
          op.coef[128 * t + 2 * i + 1] = kraus[t][i].imag();
        }
    }
    *out = std::move(op);
    return ORKAN_OK;
  }
  if (k == 1) {
    op.q[0] = qubits[0];
    op.R = ptm(1, kraus, adj);
    if (kraus.size() == 1) {
      op.L = adj ? dagger(kraus[0], 2) : kraus[0];
      op.has_L = true;
    }
    std::vector<long long> pp, qq;
    if (unitary && monomial(adj ? dagger(kraus[0], 2) : kraus[0], 2, &pp, &qq)) {
      op.kind = OP_PTM1_U;   // composes as a unitary PTM if a neighbour merges into it
      op.codes = {pp[0], pp[1], qq[0], qq[1]};
      *out = std::move(op);
      return ORKAN_OK;
    }
    if (unitary) {
      // a unitary conjugation fixes the identity and is trace preserving
      op.R[0] = 1.0;
      op.R[1] = op.R[2] = op.R[3] = op.R[4] = op.R[8] = op.R[12] = 0.0;
      op.kind = OP_PTM1_U;
    } else {
      op.kind = is_ad_pattern(op.R) ? OP_PTM1_AD : OP_PTM1;
    }
  } else {
    if (qubits[0] < qubits[1]) {
      op.q[0] = qubits[0];
      op.q[1] = qubits[1];
    } else {
      op.q[0] = qubits[1];
      op.q[1] = qubits[0];
      for (auto& K : kraus) K = swap_local_bits(K);
    }
    if (kraus.size() == 1) {
      // direct form h -> V h V^dagger (Eq. 2 with r = 1)
      const Mat V = adj ? dagger(kraus[0], 4) : kraus[0];
      op.L = V;
      op.has_L = true;
      std::vector<long long> pp, qq;
      op.kind = (unitary && monomial(V, 4, &pp, &qq)) ? OP_MONO2 : OP_U2;
      op.coef.resize(32);
      for (int i = 0; i < 16; ++i) {
        op.coef[2 * i] = V[i].real();
        op.coef[2 * i + 1] = V[i].imag();
      }
      if (op.kind == OP_MONO2) {
        op.codes = pp;
        op.codes.insert(op.codes.end(), qq.begin(), qq.end());
      }
    } else {
      const std::vector<double> R = ptm(2, kraus, adj);
      op.kind = OP_PTM2;
      op.coef.resize(256);
      for (int i = 0; i < 256; ++i) op.coef[i] = 0.25 * R[i];
    }
  }
  *out = std::move(op);
  return ORKAN_OK;
}

int make_op(orkan_ctx* h, int k, const int* qubits, const std::vector<Mat>& kraus_in, bool unitary, HostOp* out) {
  return make_op_adj(h->picture == ORKAN_OBSERVABLE, k, qubits, kraus_in, unitary, out);
}

// An AD-form op with closed-form coefficients (projectors, renormalisation).
HostOp make_ad_op(int q, const double R[16]) {
  HostOp op;
  op.nq = 1;
  op.q[0] = q;
  op.kind = OP_PTM1_AD;
  op.R.assign(R, R + 16);
  return op;
}

// Move to the logical -> physical map tgt by swapping physical bit pairs (the
// SWAP gate, a permutation pass), at most n - 1 swaps, fused by the planner.
int relabel_to(orkan_ctx* h, const int* tgt) {
  const int n = h->g.n;
  int occ[64], want[64];
  for (int q = 0; q < n; ++q) {
    occ[h->phys[q]] = q;
    want[tgt[q]] = q;
  }
  const Mat swap_gate = {1, 0, 0, 0, 0, 0, 1, 0, 0, 1, 0, 0, 0, 0, 0, 1};
  for (int p = 0; p < n; ++p) {
    if (occ[p] == want[p]) continue;
    int r = p + 1;
    while (occ[r] != want[p]) ++r;
    const int pr[2] = {p, r};
    HostOp op;
    if (int st = make_op_adj(false, 2, pr, {swap_gate}, true, &op)) return st;
    if (int st = enqueue(h, std::move(op))) return st;
    std::swap(occ[p], occ[r]);
  }
  for (int q = 0; q < n; ++q) h->phys[q] = tgt[q];
  return ORKAN_OK;
}

// Before a circuit: give the tile's m physical positions to the m logical
// qubits the circuit uses most, when the net number of ops that become
// in-tile (those that enter minus those that leave) is at least four per swap.  An incoming qubit swaps places with the least used
// outgoing one; qubits already in the tile stay where they are.
int plan_relabel(orkan_ctx* h, int count, const orkan_op* ops) {
  const int n = h->g.n, m = h->g.m;
  if (n <= m) return ORKAN_OK;
  std::vector<int64_t> use(n, 0);
  auto nq = [](const orkan_op& o) { return (o.kind == ORKAN_OP_UNITARY || o.kind == ORKAN_OP_KRAUS) ? o.k : 1; };
  for (int i = 0; i < count; ++i)
    for (int l = 0; l < nq(ops[i]) && l < 3; ++l)
      if (ops[i].qubits[l] >= 0 && ops[i].qubits[l] < n) ++use[ops[i].qubits[l]];
  std::vector<int> order(n);
  for (int q = 0; q < n; ++q) order[q] = q;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return use[a] != use[b] ? use[a] > use[b] : h->phys[a] < h->phys[b];
  });
  std::vector<char> top(n, 0);
  for (int i = 0; i < m; ++i)
    if (use[order[i]] > 0) top[order[i]] = 1;
  std::vector<int> in, out;
  for (int i = 0; i < n; ++i) {
    const int q = order[i];
    if (top[q] && h->phys[q] >= m) in.push_back(q);
  }
  for (int i = n - 1; i >= 0; --i) {
    const int q = order[i];
    if (!top[q] && h->phys[q] < m) out.push_back(q);
  }
  const size_t pairs = std::min(in.size(), out.size());
  if (pairs == 0) return ORKAN_OK;
  int tgt[64];
  for (int q = 0; q < n; ++q) tgt[q] = h->phys[q];
  for (size_t i = 0; i < pairs; ++i) std::swap(tgt[in[i]], tgt[out[i]]);
  int64_t gain = 0;
  for (int i = 0; i < count; ++i) {
    bool low_now = true, low_then = true;
    for (int l = 0; l < nq(ops[i]) && l < 3; ++l) {
      const int q = ops[i].qubits[l];
      if (q < 0 || q >= n) return ORKAN_OK;   // invalid op: leave the error to the op itself
      low_now = low_now && h->phys[q] < m;
      low_then = low_then && tgt[q] < m;
    }
    if (low_then && !low_now) ++gain;
    if (low_now && !low_then) --gain;   // ops that would leave the tile count against
  }
  if (gain < 4 * int64_t(pairs)) return ORKAN_OK;
  return relabel_to(h, tgt);
}

// Device staging space of at least `bytes` for host uploads, kept for the
// handle's lifetime; earlier uploads are stream-ordered before later ones.
int upload_space(orkan_ctx* h, size_t bytes, void** out) {
  if (bytes > h->upload_cap) {
    if (h->d_upload) {
      cudaError_t e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) return cuda_fail(e, "upload_space");
      cudaFree(h->d_upload);
      h->d_upload = nullptr;
      h->upload_cap = 0;
    }
    size_t cap = bytes < 4096 ? 4096 : bytes;
    if (cudaMalloc(&h->d_upload, cap) != cudaSuccess) {
      cudaGetLastError();
      return fail(ORKAN_ENOMEM, "cudaMalloc(upload staging) failed");
    }
    h->upload_cap = cap;
  }
  *out = h->d_upload;
  return ORKAN_OK;
}

int reduce_diag(orkan_ctx* h, int q, double out[4]) {
  int st = flush_pending(h);
  if (st != ORKAN_OK) return st;
  ORKAN_CUDA(launch_reduce_diag(h->dtype, h->d_state, h->g, q, h->d_partials, h->d_res, h->stream));
  h->n_launches += 2;
  ORKAN_CUDA(cudaMemcpyAsync(h->h_res, h->d_res, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  ORKAN_CUDA(cudaStreamSynchronize(h->stream));
  for (int i = 0; i < 4; ++i) out[i] = h->h_res[i];
  return ORKAN_OK;
}

int setup_handle(orkan_ctx* c) {
  ORKAN_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
  c->own_stream = true;
  if (cudaMalloc(&c->d_partials, sizeof(double) * 4 * kRedBlocks) != cudaSuccess)
    return fail(ORKAN_ENOMEM, "cudaMalloc(partials) failed");
  if (cudaMalloc(&c->d_res, sizeof(double) * 4) != cudaSuccess) return fail(ORKAN_ENOMEM, "cudaMalloc(res) failed");
  if (cudaMallocHost(&c->h_res, sizeof(double) * 4) != cudaSuccess)
    return fail(ORKAN_ENOMEM, "cudaMallocHost(res) failed");
  if (cudaMalloc(&c->d_err, sizeof(int32_t)) != cudaSuccess) return fail(ORKAN_ENOMEM, "cudaMalloc(err) failed");
  ORKAN_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), c->stream));
  return ORKAN_OK;
}

void release_handle(orkan_ctx* c) {
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& p : c->ev_used) {
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  for (auto e : c->ev_free) cudaEventDestroy(e);
  if (c->d_state && !c->external) cudaFree(c->d_state);
  if (c->d_upload) cudaFree(c->d_upload);
  if (c->d_partials) cudaFree(c->d_partials);
  if (c->d_res) cudaFree(c->d_res);
  if (c->d_err) cudaFree(c->d_err);
  if (c->h_res) cudaFreeHost(c->h_res);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

bool geometry(int n, int tile_log2, Geometry* g) {
  if (tile_log2 == 0) tile_log2 = 5;
  if (n < 1 || n > 24 || tile_log2 < 3 || tile_log2 > 5) return false;
  g->n = n;
  g->m = tile_log2;
  g->N = int64_t(1) << n;
  g->Nt = n > tile_log2 ? (int64_t(1) << (n - tile_log2)) : 1;
  g->ntiles = g->Nt * (g->Nt + 1) / 2;
  return true;
}

int common_alloc(int n, int dtype, int tile_log2, void* dev_ptr, size_t bytes, orkan_h* out) {
  if (!out) return fail(ORKAN_EINVAL, "null output handle");
  *out = nullptr;
  Geometry g;
  if (!valid_dtype(dtype) || !geometry(n, tile_log2, &g)) return fail(ORKAN_EINVAL, "bad n / dtype / tile_log2");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return fail(ORKAN_ENODEV, "no CUDA device");
  orkan_ctx* c = new (std::nothrow) orkan_ctx;
  if (!c) return fail(ORKAN_ENOMEM, "host allocation failed");
  c->g = g;
  c->dtype = dtype;
  for (int q = 0; q < 64; ++q) c->phys[q] = c->cap_phys[q] = q;
  c->tc_mode = dtype == DT_C64 ? 1 : 0;   // tensor-core passes for composed in-tile runs (complex64)
  c->bytes = size_t(g.ntiles) << (2 * g.m);
  c->bytes *= elem_size(dtype);
  cudaGetDevice(&c->device);
  int st = setup_handle(c);
  if (st != ORKAN_OK) {
    release_handle(c);
    return st;
  }
  if (dev_ptr) {
    if (bytes < c->bytes || (reinterpret_cast<uintptr_t>(dev_ptr) & 255) != 0) {
      release_handle(c);
      return fail(ORKAN_EINVAL, "external buffer too small or not 256-byte aligned");
    }
    c->d_state = dev_ptr;
    c->external = true;
  } else if (cudaMalloc(&c->d_state, c->bytes) != cudaSuccess) {
    cudaGetLastError();
    release_handle(c);
    return fail(ORKAN_ENOMEM, "cudaMalloc of the tiled state failed");
  }
  *out = c;
  return ORKAN_OK;
}

}  // namespace

void orkan::set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

// An instantiated circuit graph with the qubit labels it was recorded under.
struct GraphRec {
  cudaGraphExec_t exec = nullptr;
  int n = 0;
  int phys_begin[64];
  int phys_end[64];
};

// Checkpoint header (layout documented beside orkan_checkpoint_save).
namespace {
struct CkptHeader {
  char magic[8];
  int32_t version, n, tile_log2, dtype, picture, reserved;
  int32_t phys[64];
  uint64_t data_bytes;
  uint64_t checksum;
};
static_assert(sizeof(CkptHeader) <= ORKAN_CKPT_HEADER_BYTES, "checkpoint header too large");
constexpr char kCkptMagic[8] = {'O', 'R', 'K', 'A', 'N', 'C', 'K', '1'};

// FNV-1a over 64-bit little-endian words (the data is a whole number of 8-byte words).
uint64_t ckpt_checksum(const unsigned char* p, uint64_t bytes) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (uint64_t i = 0; i + 8 <= bytes; i += 8) {
    uint64_t w = 0;
    for (int b = 0; b < 8; ++b) w |= uint64_t(p[i + b]) << (8 * b);
    h = (h ^ w) * 0x100000001b3ull;
  }
  return h;
}

int ckpt_parse(const void* src, size_t bytes, CkptHeader* hd) {
  if (!src) return fail(ORKAN_EINVAL, "null checkpoint");
  if (bytes < ORKAN_CKPT_HEADER_BYTES) return fail(ORKAN_EINVAL, "checkpoint shorter than its header");
  std::memcpy(hd, src, sizeof(CkptHeader));
  if (std::memcmp(hd->magic, kCkptMagic, 8) != 0) return fail(ORKAN_EINVAL, "not an Orkan checkpoint (bad magic)");
  if (hd->version != 1) return fail(ORKAN_EINVAL, "unsupported checkpoint version");
  Geometry g;
  if (!valid_dtype(hd->dtype) || !geometry(hd->n, hd->tile_log2, &g))
    return fail(ORKAN_EINVAL, "checkpoint header: bad n / dtype / tile_log2");
  if (hd->picture != ORKAN_STATE && hd->picture != ORKAN_OBSERVABLE)
    return fail(ORKAN_EINVAL, "checkpoint header: bad picture");
  std::vector<char> seen(hd->n, 0);
  for (int q = 0; q < hd->n; ++q) {
    if (hd->phys[q] < 0 || hd->phys[q] >= hd->n || seen[hd->phys[q]])
      return fail(ORKAN_EINVAL, "checkpoint header: labels are not a permutation");
    seen[hd->phys[q]] = 1;
  }
  const uint64_t want = (uint64_t(g.ntiles) << (2 * g.m)) * elem_size(hd->dtype);
  if (hd->data_bytes != want) return fail(ORKAN_EINVAL, "checkpoint header: data size does not match n / dtype / tile_log2");
  if (bytes < ORKAN_CKPT_HEADER_BYTES + want) return fail(ORKAN_EINVAL, "checkpoint truncated");
  const unsigned char* data = static_cast<const unsigned char*>(src) + ORKAN_CKPT_HEADER_BYTES;
  if (ckpt_checksum(data, want) != hd->checksum) return fail(ORKAN_EINVAL, "checkpoint data checksum mismatch");
  return ORKAN_OK;
}
}  // namespace

// =================================================================== C ABI
extern "C" {

const char* orkan_strerror(int status) {
  switch (status) {
    case ORKAN_OK: return "ok";
    case ORKAN_EINVAL: return "invalid argument";
    case ORKAN_ENOMEM: return "out of memory";
    case ORKAN_ECUDA: return "CUDA error";
    case ORKAN_EZEROPROB: return "zero-probability outcome";
    case ORKAN_EPICTURE: return "operation not defined in this picture";
    case ORKAN_ENODEV: return "no CUDA device";
    case ORKAN_ETIMEOUT: return "a bounded device wait ran out";
  }
  return "unknown status";
}

const char* orkan_last_error(void) { return g_last_error.c_str(); }

size_t orkan_bytes(int n, int dtype, int tile_log2) {
  Geometry g;
  if (!valid_dtype(dtype) || !geometry(n, tile_log2, &g)) return 0;
  return (size_t(g.ntiles) << (2 * g.m)) * size_t(elem_size(dtype));
}

int64_t orkan_num_tiles(int n, int tile_log2) {
  Geometry g;
  if (!geometry(n, tile_log2, &g)) return -1;
  return g.ntiles;
}

int64_t orkan_element_offset(int n, int tile_log2, int64_t i, int64_t j, int* conj) {
  Geometry g;
  if (!geometry(n, tile_log2, &g) || i < 0 || j < 0 || i >= g.N || j >= g.N) return -1;
  int cj = 0;
  if (i < j) {
    std::swap(i, j);
    cj = 1;
  }
  if (conj) *conj = cj;
  const int64_t ti = i >> g.m, tj = j >> g.m, M = int64_t(1) << g.m;
  return ((ti * (ti + 1) / 2 + tj) << (2 * g.m)) + (i & (M - 1)) * M + (j & (M - 1));
}

uint64_t orkan_insert_bits(uint64_t s, uint64_t a, int k, const int* pos) {
  // Subroutine 1: for each active position (ascending), split the index there
  // and drop bit l of a into the gap.
  uint64_t global = s;
  for (int l = 0; l < k; ++l) {
    const int p = pos[l];
    const uint64_t right = ((uint64_t(1) << p) - 1) & global;
    uint64_t left = (global >> p) << 1;
    left |= (a >> l) & 1;
    left <<= p;
    global = left | right;
  }
  return global;
}

int orkan_ptm(int k, int r, const double* K, int adjoint, double* out) {
  if (k < 1 || k > 2 || r < 1 || r > (1 << (2 * k)) || !K || !out) return fail(ORKAN_EINVAL, "bad ptm arguments");
  const int d = 1 << k;
  std::vector<Mat> kraus;
  for (int a = 0; a < r; ++a) kraus.push_back(read_mat(K + 2 * d * d * a, d));
  const std::vector<double> R = ptm(k, kraus, adjoint != 0);
  std::copy(R.begin(), R.end(), out);
  return ORKAN_OK;
}

int orkan_alloc(int n, int dtype, int tile_log2, orkan_h* out) {
  return common_alloc(n, dtype, tile_log2, nullptr, 0, out);
}

int orkan_alloc_external(int n, int dtype, int tile_log2, void* dev_ptr, size_t bytes, orkan_h* out) {
  if (!dev_ptr) return fail(ORKAN_EINVAL, "null device pointer");
  // the kernels move 16-byte granules and bulk-prefetch 8 KiB tiles
  if (reinterpret_cast<uintptr_t>(dev_ptr) & 255u) return fail(ORKAN_EINVAL, "device pointer is not 256-byte aligned");
  return common_alloc(n, dtype, tile_log2, dev_ptr, bytes, out);
}

int orkan_free(orkan_h h) {
  if (!h) return ORKAN_OK;
  h->pending.clear();
  h->held.clear();
  release_handle(h);
  return ORKAN_OK;
}

int orkan_set_stream(orkan_h h, void* cuda_stream) {
  if (int st = check_blocking(h)) return st;
  if (int st = flush_pending(h)) return st;
  if (h->own_stream && h->stream) {
    ORKAN_CUDA(cudaStreamSynchronize(h->stream));
    cudaStreamDestroy(h->stream);
  }
  h->own_stream = false;
  h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  return ORKAN_OK;
}

int orkan_set_tensor(orkan_h h, int mode) {
  if (int st = check_handle(h)) return st;
  if (mode < 0 || mode > 2) return fail(ORKAN_EINVAL, "mode must be 0, 1 or 2");
  if (int st = flush_pending(h)) return st;
  h->tc_mode = mode;
  return ORKAN_OK;
}

int orkan_set_fusion(orkan_h h, int max_ops, int compose) {
  if (int st = check_handle(h)) return st;
  if (max_ops < 1 || max_ops > kMaxOps) return fail(ORKAN_EINVAL, "max_ops must be in 1..16");
  if (int st = flush_pending(h)) return st;
  h->fusion = max_ops;
  h->compose = compose != 0;
  return ORKAN_OK;
}

int orkan_get_info(orkan_h h, int* n, int* dtype, int* tile_log2, int* picture) {
  if (int st = check_handle(h)) return st;
  if (n) *n = h->g.n;
  if (dtype) *dtype = h->dtype;
  if (tile_log2) *tile_log2 = h->g.m;
  if (picture) *picture = h->picture;
  return ORKAN_OK;
}

void* orkan_device_ptr(orkan_h h) { return h ? h->d_state : nullptr; }

int orkan_init_state(orkan_h h, int kind, const double* data) {
  if (int st = check_blocking(h)) return st;
  h->pending.clear();
  h->held.clear();
  reset_labels(h);
  h->picture = ORKAN_STATE;
  switch (kind) {
    case ORKAN_INIT_ZERO:
      ORKAN_CUDA(launch_zero(h->dtype, h->d_state, h->g, h->stream));
      ORKAN_CUDA(launch_set_diag(h->dtype, h->d_state, h->g, 0, 1.0, h->stream));
      h->n_launches += 2;
      return ORKAN_OK;
    case ORKAN_INIT_MAXMIXED:
      ORKAN_CUDA(launch_zero(h->dtype, h->d_state, h->g, h->stream));
      ORKAN_CUDA(launch_fill_diag(h->dtype, h->d_state, h->g, 1.0 / double(h->g.N), h->stream));
      h->n_launches += 2;
      return ORKAN_OK;
    case ORKAN_INIT_DENSE:
    case ORKAN_INIT_PURE: {
      if (!data) return fail(ORKAN_EINVAL, "data required");
      const size_t count = kind == ORKAN_INIT_DENSE ? size_t(h->g.N) * size_t(h->g.N) : size_t(h->g.N);
      void* tmp = nullptr;
      if (int st = upload_space(h, count * 16, &tmp)) return st;
      ORKAN_CUDA(cudaMemcpyAsync(tmp, data, count * 16, cudaMemcpyHostToDevice, h->stream));
      if (kind == ORKAN_INIT_DENSE)
        ORKAN_CUDA(launch_from_dense(h->dtype, h->d_state, h->g, static_cast<const double*>(tmp), h->stream));
      else
        ORKAN_CUDA(launch_from_pure(h->dtype, h->d_state, h->g, static_cast<const double*>(tmp), h->stream));
      h->n_launches += 1;
      return ORKAN_OK;
    }
  }
  return fail(ORKAN_EINVAL, "unknown init kind");
}

int orkan_set_picture(orkan_h h, int picture) {
  if (int st = check_handle(h)) return st;
  if (picture != ORKAN_STATE && picture != ORKAN_OBSERVABLE) return fail(ORKAN_EINVAL, "bad picture");
  if (int st = flush_pending(h)) return st;
  h->picture = picture;
  return ORKAN_OK;
}

int orkan_init_observable(orkan_h h, int nterms, const char* paulis, const double* coeffs) {
  if (int st = check_blocking(h)) return st;
  if (nterms < 0 || (nterms > 0 && (!paulis || !coeffs))) return fail(ORKAN_EINVAL, "bad Pauli sum");
  const int n = h->g.n;
  struct Term {
    uint64_t x, z, y, ny;
    double c;
  };
  std::vector<Term> terms;
  for (int t = 0; t < nterms; ++t) {
    Term tm{0, 0, 0, 0, coeffs[t]};
    for (int l = 0; l < n; ++l) {
      const char ch = paulis[size_t(t) * n + l];
      const uint64_t bit = uint64_t(1) << l;
      if (ch == 'I') continue;
      if (ch == 'X') tm.x |= bit;
      else if (ch == 'Y') { tm.x |= bit; tm.y |= bit; tm.ny += 1; }
      else if (ch == 'Z') tm.z |= bit;
      else return fail(ORKAN_EINVAL, "Pauli characters must be I, X, Y or Z");
    }
    terms.push_back(tm);
  }
  std::stable_sort(terms.begin(), terms.end(), [](const Term& a, const Term& b) { return a.x < b.x; });
  h->pending.clear();
  h->held.clear();
  reset_labels(h);
  h->picture = ORKAN_OBSERVABLE;
  ORKAN_CUDA(launch_zero(h->dtype, h->d_state, h->g, h->stream));
  h->n_launches += 1;
  if (terms.empty()) return ORKAN_OK;
  std::vector<uint64_t> masks;
  std::vector<double> cs;
  for (const auto& t : terms) {
    masks.insert(masks.end(), {t.x, t.z, t.y, t.ny});
    cs.push_back(t.c);
  }
  void* stage = nullptr;
  const size_t mbytes = masks.size() * 8, cbytes = cs.size() * 8;
  if (int st = upload_space(h, mbytes + cbytes, &stage)) return st;
  uint64_t* dm = static_cast<uint64_t*>(stage);
  double* dc = reinterpret_cast<double*>(static_cast<char*>(stage) + mbytes);
  ORKAN_CUDA(cudaMemcpyAsync(dm, masks.data(), mbytes, cudaMemcpyHostToDevice, h->stream));
  ORKAN_CUDA(cudaMemcpyAsync(dc, cs.data(), cbytes, cudaMemcpyHostToDevice, h->stream));
  // masks / cs are host temporaries: the copies must have read them before return
  ORKAN_CUDA(launch_pauli_sum(h->dtype, h->d_state, h->g, int(terms.size()), dm, dc, h->stream));
  ORKAN_CUDA(cudaStreamSynchronize(h->stream));
  h->n_launches += 1;
  return ORKAN_OK;
}

int orkan_load_tiled(orkan_h h, const void* host_src, int picture) {
  if (int st = check_blocking(h)) return st;
  if (!host_src || (picture != ORKAN_STATE && picture != ORKAN_OBSERVABLE)) return fail(ORKAN_EINVAL, "bad args");
  h->pending.clear();
  h->held.clear();
  reset_labels(h);
  h->picture = picture;
  ORKAN_CUDA(cudaMemcpyAsync(h->d_state, host_src, h->bytes, cudaMemcpyHostToDevice, h->stream));
  ORKAN_CUDA(cudaStreamSynchronize(h->stream));
  return ORKAN_OK;
}

int orkan_load_tiled_async(orkan_h h, const void* host_src, int picture) {
  if (int st = check_blocking(h)) return st;
  if (!host_src || (picture != ORKAN_STATE && picture != ORKAN_OBSERVABLE)) return fail(ORKAN_EINVAL, "bad args");
  h->pending.clear();
  h->held.clear();
  reset_labels(h);
  h->picture = picture;
  ORKAN_CUDA(cudaMemcpyAsync(h->d_state, host_src, h->bytes, cudaMemcpyHostToDevice, h->stream));
  return ORKAN_OK;
}

int orkan_store_tiled(orkan_h h, void* host_dst) {
  if (int st = check_blocking(h)) return st;
  if (!host_dst) return fail(ORKAN_EINVAL, "null destination");
  if (!labels_identity(h)) {   // the stored layout is the logical one
    int id[64];
    for (int q = 0; q < 64; ++q) id[q] = q;
    if (int st = relabel_to(h, id)) return st;
  }
  if (int st = flush_pending(h)) return st;
  ORKAN_CUDA(cudaMemcpyAsync(host_dst, h->d_state, h->bytes, cudaMemcpyDeviceToHost, h->stream));
  ORKAN_CUDA(cudaStreamSynchronize(h->stream));
  return ORKAN_OK;
}

// ------------------------------------------------------------------ checkpoints

size_t orkan_checkpoint_bytes(orkan_h h) { return h ? ORKAN_CKPT_HEADER_BYTES + h->bytes : 0; }

int orkan_checkpoint_save(orkan_h h, void* host_dst, size_t cap) {
  if (int st = check_blocking(h)) return st;
  if (!host_dst) return fail(ORKAN_EINVAL, "null destination");
  if (cap < ORKAN_CKPT_HEADER_BYTES + h->bytes) return fail(ORKAN_EINVAL, "destination smaller than orkan_checkpoint_bytes");
  if (int st = flush_pending(h)) return st;
  unsigned char* data = static_cast<unsigned char*>(host_dst) + ORKAN_CKPT_HEADER_BYTES;
  ORKAN_CUDA(cudaMemcpyAsync(data, h->d_state, h->bytes, cudaMemcpyDeviceToHost, h->stream));
  ORKAN_CUDA(cudaStreamSynchronize(h->stream));
  CkptHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, kCkptMagic, 8);
  hd.version = 1;
  hd.n = h->g.n;
  hd.tile_log2 = h->g.m;
  hd.dtype = h->dtype;
  hd.picture = h->picture;
  for (int q = 0; q < 64; ++q) hd.phys[q] = h->phys[q];
  hd.data_bytes = h->bytes;
  hd.checksum = ckpt_checksum(data, h->bytes);
  std::memset(host_dst, 0, ORKAN_CKPT_HEADER_BYTES);
  std::memcpy(host_dst, &hd, sizeof(hd));
  return ORKAN_OK;
}

int orkan_checkpoint_load(orkan_h h, const void* host_src, size_t bytes) {
  if (int st = check_blocking(h)) return st;
  CkptHeader hd;
  if (int st = ckpt_parse(host_src, bytes, &hd)) return st;
  if (hd.n != h->g.n || hd.tile_log2 != h->g.m || hd.dtype != h->dtype)
    return fail(ORKAN_EINVAL, "checkpoint is for n=" + std::to_string(hd.n) + " tile_log2=" +
                                  std::to_string(hd.tile_log2) + " dtype=" + std::to_string(hd.dtype) +
                                  ", the handle has n=" + std::to_string(h->g.n) + " tile_log2=" +
                                  std::to_string(h->g.m) + " dtype=" + std::to_string(h->dtype));
  h->pending.clear();
  h->held.clear();
  const unsigned char* data = static_cast<const unsigned char*>(host_src) + ORKAN_CKPT_HEADER_BYTES;
  ORKAN_CUDA(cudaMemcpyAsync(h->d_state, data, h->bytes, cudaMemcpyHostToDevice, h->stream));
  ORKAN_CUDA(cudaStreamSynchronize(h->stream));
  reset_labels(h);
  for (int q = 0; q < h->g.n; ++q) h->phys[q] = hd.phys[q];
  h->picture = hd.picture;
  return ORKAN_OK;
}

int orkan_checkpoint_inspect(const void* host_src, size_t bytes, int* n, int* dtype, int* tile_log2, int* picture) {
  CkptHeader hd;
  if (int st = ckpt_parse(host_src, bytes, &hd)) return st;
  if (n) *n = hd.n;
  if (dtype) *dtype = hd.dtype;
  if (tile_log2) *tile_log2 = hd.tile_log2;
  if (picture) *picture = hd.picture;
  return ORKAN_OK;
}

int orkan_apply_unitary(orkan_h h, int k, const int* qubits, const double* U) {
  if (int st = check_handle(h)) return st;
  if (int st = check_qubits(h, k, qubits)) return st;
  if (!U) return fail(ORKAN_EINVAL, "null matrix");
  int pq[3];
  map_qubits(h, k, qubits, pq);
  HostOp op;
  if (int st = make_op(h, k, pq, {read_mat(U, 1 << k)}, true, &op)) return st;
  return enqueue(h, std::move(op));
}

int orkan_apply_kraus(orkan_h h, int k, const int* qubits, int r, const double* K) {
  if (int st = check_handle(h)) return st;
  if (int st = check_qubits(h, k, qubits)) return st;
  if (!K || r < 1 || r > (1 << (2 * k))) return fail(ORKAN_EINVAL, "need 1 <= r <= 4^k Kraus operators");
  if (k == 3 && r > kK3MaxTerms) return fail(ORKAN_EINVAL, "three-qubit Kraus sets are limited to 16 operators");
  const int d = 1 << k;
  std::vector<Mat> kraus;
  for (int a = 0; a < r; ++a) kraus.push_back(read_mat(K + 2 * d * d * a, d));
  int pq[3];
  map_qubits(h, k, qubits, pq);
  HostOp op;
  if (int st = make_op(h, k, pq, kraus, false, &op)) return st;
  return enqueue(h, std::move(op));
}

static int named_channel(orkan_h h, int q, const std::vector<Mat>& kraus) {
  if (int st = check_handle(h)) return st;
  if (int st = check_qubits(h, 1, &q)) return st;
  const int pq = h->phys[q];
  HostOp op;
  if (int st = make_op(h, 1, &pq, kraus, false, &op)) return st;
  op.kind = OP_PTM1_AD;   // diagonal / amplitude-mixing structure holds exactly for these sets
  return enqueue(h, std::move(op));
}

int orkan_depolarize(orkan_h h, int q, double p) {
  if (!(p >= 0.0 && p <= 1.0)) return fail(ORKAN_EINVAL, "p must be in [0, 1]");
  if (int st = check_handle(h)) return st;
  if (int st = check_qubits(h, 1, &q)) return st;
  // Kraus sqrt(1-p) I, sqrt(p/3) {X, Y, Z} (Sec. IV-A) have the self-adjoint
  // transfer matrix diag(1, f, f, f), f = 1 - 4p/3, used in closed form.
  const double f = 1.0 - 4.0 * p / 3.0;
  const double R[16] = {1, 0, 0, 0, 0, f, 0, 0, 0, 0, f, 0, 0, 0, 0, f};
  return enqueue(h, make_ad_op(h->phys[q], R));
}

int orkan_dephase(orkan_h h, int q, double p) {
  if (!(p >= 0.0 && p <= 1.0)) return fail(ORKAN_EINVAL, "p must be in [0, 1]");
  const double a = std::sqrt(1.0 - p), b = std::sqrt(p);
  return named_channel(h, q, {{a, 0, 0, a}, {b, 0, 0, -b}});
}

int orkan_amplitude_damp(orkan_h h, int q, double gamma) {
  if (!(gamma >= 0.0 && gamma <= 1.0)) return fail(ORKAN_EINVAL, "gamma must be in [0, 1]");
  const double s = std::sqrt(1.0 - gamma), g = std::sqrt(gamma);
  return named_channel(h, q, {{1, 0, 0, s}, {0, g, 0, 0}});
}

int orkan_measure(orkan_h h, int q, double u, int* outcome, double* prob) {
  if (int st = check_blocking(h)) return st;
  if (h->picture != ORKAN_STATE) return fail(ORKAN_EPICTURE, "measure needs a state handle (use orkan_project)");
  if (int st = check_qubits(h, 1, &q)) return st;
  if (!(u >= 0.0 && u < 1.0)) return fail(ORKAN_EINVAL, "u must be in [0, 1)");
  double r[4];
  if (int st = reduce_diag(h, h->phys[q], r)) return st;
  const double p0 = r[2], p1 = r[3], tot = p0 + p1;
  if (!(tot > 0.0)) return fail(ORKAN_EZEROPROB, "both outcomes have zero probability");
  const int b = (u * tot < p0) ? 0 : 1;
  const double pb = b ? p1 : p0;
  if (!(pb > 1e-300)) return fail(ORKAN_EZEROPROB, "selected outcome has zero probability");
  const double s = 1.0 / pb;
  // transfer matrix of Pi_b . Pi_b / p_b
  const double sg = b ? -0.5 * s : 0.5 * s;
  const double R[16] = {0.5 * s, 0, 0, sg, 0, 0, 0, 0, 0, 0, 0, 0, sg, 0, 0, 0.5 * s};
  if (int st = enqueue(h, make_ad_op(h->phys[q], R))) return st;
  if (outcome) *outcome = b;
  if (prob) *prob = pb / tot;
  return ORKAN_OK;
}

int orkan_project(orkan_h h, int q, int outcome) {
  if (int st = check_handle(h)) return st;
  if (int st = check_qubits(h, 1, &q)) return st;
  if (outcome != 0 && outcome != 1) return fail(ORKAN_EINVAL, "outcome must be 0 or 1");
  const double sg = outcome ? -0.5 : 0.5;
  const double R[16] = {0.5, 0, 0, sg, 0, 0, 0, 0, 0, 0, 0, 0, sg, 0, 0, 0.5};
  return enqueue(h, make_ad_op(h->phys[q], R));
}

// ------------------------------------------------------------------ packed column-major layout
size_t orkan_packed_bytes(int n, int dtype) {
  if (n < 1 || n > 24 || (dtype != DT_C128 && dtype != DT_C64 && dtype != DT_DF64)) return 0;
  const int64_t N = int64_t(1) << n;
  return size_t(N * (N + 1) / 2) * size_t(elem_size(dtype));
}

int64_t orkan_packed_offset(int n, int64_t i, int64_t j, int* conj) {
  if (n < 1 || n > 24) return -1;
  const int64_t N = int64_t(1) << n;
  if (i < 0 || j < 0 || i >= N || j >= N) return -1;
  const bool cj = i < j;
  if (conj) *conj = cj ? 1 : 0;
  const int64_t p = cj ? j : i, q = cj ? i : j;
  return q * N - q * (q - 1) / 2 + (p - q);
}

namespace {
int packed_args(const void* dev, int n, int dtype) {
  if (!dev) return fail(ORKAN_EINVAL, "null packed array");
  if (orkan_packed_bytes(n, dtype) == 0) return fail(ORKAN_EINVAL, "bad n or dtype");
  return ORKAN_OK;
}

int packed_run(void* dev, int n, int dtype, const HostOp& op, void* stream) {
  PackedDesc d;
  std::memset(&d, 0, sizeof(d));
  d.N = int64_t(1) << n;
  d.k = op.nq;
  d.q[0] = op.q[0];
  d.q[1] = op.nq == 2 ? op.q[1] : 0;
  if (op.nq == 1) {
    if (!op.codes.empty()) {
      d.kind = OP_MONO1;
      for (int i = 0; i < 4; ++i) std::memcpy(&d.coef[i], &op.codes[i], 8);
    } else {
      d.kind = op.kind;
      pack_op_coefs(dtype, op.kind, coef_1q(op.kind, op.R), d.coef);
    }
  } else {
    if (op.kind != OP_U2 && op.kind != OP_MONO2)
      return fail(ORKAN_EINVAL, "packed layout: two-qubit maps must be unitary (one Kraus operator)");
    d.kind = op.kind;
    pack_op_coefs(dtype, op.kind, std::vector<double>(op.coef.begin(), op.coef.begin() + 32), d.coef);
    for (size_t i = 0; i < op.codes.size(); ++i) std::memcpy(&d.coef[32 + i], &op.codes[i], 8);
  }
  const int64_t S = d.N >> d.k;
  d.n_blocks = S * (S + 1) / 2;
  const cudaError_t e = launch_packed(dtype, dev, d, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? ORKAN_OK : cuda_fail(e, "packed op");
}

int packed_kraus(void* dev, int n, int dtype, int picture, int k, const int* qubits, const std::vector<Mat>& kraus,
                 bool unitary, void* stream) {
  if (int st = packed_args(dev, n, dtype)) return st;
  if (picture != ORKAN_STATE && picture != ORKAN_OBSERVABLE) return fail(ORKAN_EINVAL, "bad picture");
  if (k > 2) return fail(ORKAN_EINVAL, "packed layout: k must be 1 or 2");
  if (int st = check_qubits_n(n, k, qubits)) return st;
  HostOp op;
  if (int st = make_op_adj(picture == ORKAN_OBSERVABLE, k, qubits, kraus, unitary, &op)) return st;
  return packed_run(dev, n, dtype, op, stream);
}
}  // namespace

int orkan_packed_apply_unitary(void* dev_packed, int n, int dtype, int picture, int k, const int* qubits,
                               const double* U, void* cuda_stream) {
  if (!U || k < 1 || k > 2) return fail(ORKAN_EINVAL, "packed layout: need k = 1 or 2 and a matrix");
  return packed_kraus(dev_packed, n, dtype, picture, k, qubits, {read_mat(U, 1 << k)}, true, cuda_stream);
}

int orkan_packed_apply_kraus(void* dev_packed, int n, int dtype, int picture, int k, const int* qubits, int r,
                             const double* K, void* cuda_stream) {
  if (!K || k < 1 || k > 2 || r < 1 || r > (1 << (2 * k))) return fail(ORKAN_EINVAL, "bad Kraus arguments");
  const int d = 1 << k;
  std::vector<Mat> kraus;
  for (int a = 0; a < r; ++a) kraus.push_back(read_mat(K + 2 * d * d * a, d));
  return packed_kraus(dev_packed, n, dtype, picture, k, qubits, kraus, false, cuda_stream);
}

int orkan_packed_depolarize(void* dev_packed, int n, int dtype, int q, double p, void* cuda_stream) {
  if (!(p >= 0.0 && p <= 1.0)) return fail(ORKAN_EINVAL, "p must be in [0, 1]");
  if (int st = packed_args(dev_packed, n, dtype)) return st;
  if (int st = check_qubits_n(n, 1, &q)) return st;
  const double f = 1.0 - 4.0 * p / 3.0;   // self-adjoint: the same in both pictures
  const double R[16] = {1, 0, 0, 0, 0, f, 0, 0, 0, 0, f, 0, 0, 0, 0, f};
  return packed_run(dev_packed, n, dtype, make_ad_op(q, R), cuda_stream);
}

int orkan_packed_from_tiled(orkan_h h, void* dev_packed) {
  if (int st = check_handle(h)) return st;
  if (!dev_packed) return fail(ORKAN_EINVAL, "null packed array");
  if (!labels_identity(h)) {
    int id[64];
    for (int q = 0; q < 64; ++q) id[q] = q;
    if (int st = relabel_to(h, id)) return st;
  }
  if (int st = flush_pending(h)) return st;
  ORKAN_CUDA(launch_packed_convert(h->dtype, dev_packed, h->d_state, h->g, 1, h->stream));
  return ORKAN_OK;
}

int orkan_packed_to_tiled(orkan_h h, const void* dev_packed) {
  if (int st = check_handle(h)) return st;
  if (!dev_packed) return fail(ORKAN_EINVAL, "null packed array");
  if (int st = flush_pending(h)) return st;
  reset_labels(h);
  ORKAN_CUDA(launch_packed_convert(h->dtype, const_cast<void*>(dev_packed), h->d_state, h->g, 0, h->stream));
  return ORKAN_OK;
}

int orkan_run_circuit(orkan_h h, int count, const orkan_op* ops, int* outcomes, double* probs, int* done) {
  if (int st = check_handle(h)) return st;
  if (count < 0 || (count > 0 && !ops)) return fail(ORKAN_EINVAL, "bad op list");
  if (h->auto_relabel)
    if (int rst = plan_relabel(h, count, ops)) return rst;
  int nmeas = 0, i = 0, st = ORKAN_OK;
  for (; i < count && st == ORKAN_OK; ++i) {
    const orkan_op& o = ops[i];
    switch (o.kind) {
      case ORKAN_OP_UNITARY: st = orkan_apply_unitary(h, o.k, o.qubits, o.mats); break;
      case ORKAN_OP_KRAUS: st = orkan_apply_kraus(h, o.k, o.qubits, o.r, o.mats); break;
      case ORKAN_OP_DEPOLARIZE: st = orkan_depolarize(h, o.qubits[0], o.param); break;
      case ORKAN_OP_DEPHASE: st = orkan_dephase(h, o.qubits[0], o.param); break;
      case ORKAN_OP_AMPDAMP: st = orkan_amplitude_damp(h, o.qubits[0], o.param); break;
      case ORKAN_OP_MEASURE: {
        int b = 0;
        double pr = 0.0;
        st = orkan_measure(h, o.qubits[0], o.param, &b, &pr);
        if (st == ORKAN_OK) {
          if (outcomes) outcomes[nmeas] = b;
          if (probs) probs[nmeas] = pr;
          ++nmeas;
        }
        break;
      }
      case ORKAN_OP_PROJECT: st = orkan_project(h, o.qubits[0], o.outcome); break;
      default: st = fail(ORKAN_EINVAL, "unknown op kind");
    }
  }
  // a circuit ends its held single-qubit ops: they join the pending pass (not
  // yet launched), so a later call cannot absorb them and a circuit's passes
  // are the same whether it is run directly or recorded and replayed
  if (st == ORKAN_OK && !h->held.empty()) st = release_held(h);
  if (done) *done = st == ORKAN_OK ? i : i - 1;
  return st;
}

int orkan_trace(orkan_h h, double* re, double* im) {
  if (int st = check_blocking(h)) return st;
  double r[4];
  if (int st = reduce_diag(h, -1, r)) return st;
  if (re) *re = r[0];
  if (im) *im = r[1];
  return ORKAN_OK;
}

int orkan_expect_pauli(orkan_h h, const char* pauli, double* out) {
  if (int st = check_blocking(h)) return st;
  if (!pauli || !out) return fail(ORKAN_EINVAL, "null argument");
  uint64_t x = 0, z = 0, y = 0;
  int ny = 0;
  for (int l = 0; l < h->g.n; ++l) {
    const char ch = pauli[l];
    const uint64_t bit = uint64_t(1) << h->phys[l];   // character l acts on logical qubit l
    if (ch == 'I') continue;
    if (ch == 'X') x |= bit;
    else if (ch == 'Y') { x |= bit; y |= bit; ++ny; }
    else if (ch == 'Z') z |= bit;
    else return fail(ORKAN_EINVAL, "Pauli characters must be I, X, Y or Z");
  }
  if (pauli[h->g.n] != '\0') return fail(ORKAN_EINVAL, "Pauli string must have n characters");
  if (int st = flush_pending(h)) return st;
  ORKAN_CUDA(launch_reduce_pauli(h->dtype, h->d_state, h->g, x, z, y, h->d_partials, h->d_res, h->stream));
  h->n_launches += 2;
  ORKAN_CUDA(cudaMemcpyAsync(h->h_res, h->d_res, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  ORKAN_CUDA(cudaStreamSynchronize(h->stream));
  const double sr = h->h_res[0], si = h->h_res[1];
  // tr(P H) = i^{nY} S
  switch (ny & 3) {
    case 0: *out = sr; break;
    case 1: *out = -si; break;
    case 2: *out = -sr; break;
    default: *out = si; break;
  }
  return ORKAN_OK;
}

int orkan_expect(orkan_h rho, orkan_h O, double* out) {
  if (int st = check_blocking(rho)) return st;
  if (int st = check_blocking(O)) return st;
  if (!out) return fail(ORKAN_EINVAL, "null output");
  if (rho->g.n != O->g.n || rho->g.m != O->g.m || rho->dtype != O->dtype)
    return fail(ORKAN_EINVAL, "operands differ in n, tile size or dtype");
  if (O != rho && !std::equal(rho->phys, rho->phys + rho->g.n, O->phys))
    if (int st = relabel_to(O, rho->phys)) return st;   // same physical layout for the tile-wise products
  if (int st = flush_pending(O)) return st;
  if (O != rho) ORKAN_CUDA(cudaStreamSynchronize(O->stream));
  if (int st = flush_pending(rho)) return st;
  ORKAN_CUDA(launch_reduce_expect(rho->dtype, rho->d_state, O->d_state, rho->g, rho->d_partials, rho->d_res,
                                  rho->stream));
  rho->n_launches += 2;
  ORKAN_CUDA(cudaMemcpyAsync(rho->h_res, rho->d_res, sizeof(double), cudaMemcpyDeviceToHost, rho->stream));
  ORKAN_CUDA(cudaStreamSynchronize(rho->stream));
  *out = rho->h_res[0];
  return ORKAN_OK;
}

int orkan_to_dense(orkan_h h, double* out) {
  if (int st = check_blocking(h)) return st;
  if (!out) return fail(ORKAN_EINVAL, "null output");
  if (int st = flush_pending(h)) return st;
  const size_t bytes = size_t(h->g.N) * size_t(h->g.N) * 16;
  double* tmp = nullptr;
  if (cudaMalloc(&tmp, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(ORKAN_ENOMEM, "cudaMalloc(dense) failed");
  }
  const bool ident = labels_identity(h);
  std::vector<double> phys_dense;
  if (!ident) phys_dense.resize(size_t(h->g.N) * size_t(h->g.N) * 2);
  cudaError_t e = launch_to_dense(h->dtype, h->d_state, h->g, tmp, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ident ? out : phys_dense.data(), tmp, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "to_dense");
  if (!ident) {   // logical (i, j) sits at the physical indices of its bits
    const int64_t N = h->g.N;
    std::vector<int64_t> pi(N);
    for (int64_t i = 0; i < N; ++i) pi[i] = int64_t(phys_index(h, uint64_t(i)));
    for (int64_t i = 0; i < N; ++i)
      for (int64_t j = 0; j < N; ++j) {
        const size_t src = (size_t(pi[i]) * N + size_t(pi[j])) * 2, dst = (size_t(i) * N + size_t(j)) * 2;
        out[dst] = phys_dense[src];
        out[dst + 1] = phys_dense[src + 1];
      }
  }
  h->n_launches += 1;
  return ORKAN_OK;
}

int orkan_get_elements(orkan_h h, int64_t count, const int64_t* rows, const int64_t* cols, double* out) {
  if (int st = check_blocking(h)) return st;
  if (count < 0 || (count > 0 && (!rows || !cols || !out))) return fail(ORKAN_EINVAL, "bad element list");
  if (count == 0) return flush_pending(h);
  for (int64_t t = 0; t < count; ++t)
    if (rows[t] < 0 || rows[t] >= h->g.N || cols[t] < 0 || cols[t] >= h->g.N)
      return fail(ORKAN_EINVAL, "element index out of range");
  if (int st = flush_pending(h)) return st;
  std::vector<int64_t> prow, pcol;
  if (!labels_identity(h)) {
    prow.resize(count);
    pcol.resize(count);
    for (int64_t t = 0; t < count; ++t) {
      prow[t] = int64_t(phys_index(h, uint64_t(rows[t])));
      pcol[t] = int64_t(phys_index(h, uint64_t(cols[t])));
    }
    rows = prow.data();
    cols = pcol.data();
  }
  int64_t* d_idx = nullptr;
  double* d_out = nullptr;
  if (cudaMalloc(&d_idx, size_t(count) * 16) != cudaSuccess || cudaMalloc(&d_out, size_t(count) * 16) != cudaSuccess) {
    cudaGetLastError();
    if (d_idx) cudaFree(d_idx);
    return fail(ORKAN_ENOMEM, "cudaMalloc(gather) failed");
  }
  cudaError_t e = cudaMemcpyAsync(d_idx, rows, size_t(count) * 8, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_idx + count, cols, size_t(count) * 8, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = launch_gather(h->dtype, h->d_state, h->g, count, d_idx, d_idx + count, d_out, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, size_t(count) * 16, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaFree(d_idx);
  cudaFree(d_out);
  if (e != cudaSuccess) return cuda_fail(e, "get_elements");
  h->n_launches += 1;
  return ORKAN_OK;
}

int orkan_flush(orkan_h h) {
  if (int st = check_handle(h)) return st;
  return flush_pending(h);
}

int orkan_sync(orkan_h h) {
  if (int st = check_blocking(h)) return st;
  if (int st = flush_pending(h)) return st;
  ORKAN_CUDA(cudaStreamSynchronize(h->stream));
  if (h->tc_mode) {
    int32_t e = 0;
    ORKAN_CUDA(cudaMemcpy(&e, h->d_err, sizeof(e), cudaMemcpyDeviceToHost));
    if (e) {
      ORKAN_CUDA(cudaMemset(h->d_err, 0, sizeof(e)));
      return fail(ORKAN_ETIMEOUT, "tensor-core pass: an mbarrier wait ran out (the operator is undefined)");
    }
  }
  return ORKAN_OK;
}

int orkan_capture_begin(orkan_h h) {
  if (int st = check_blocking(h)) return st;
  if (!h->stream) return fail(ORKAN_EINVAL, "graph capture needs a non-default stream (see orkan_set_stream)");
  if (int st = flush_pending(h)) return st;
  ORKAN_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  h->capturing = true;
  std::copy(h->phys, h->phys + 64, h->cap_phys);
  return ORKAN_OK;
}

int orkan_capture_end(orkan_h h, void** graph) {
  if (int st = check_handle(h)) return st;
  if (!h->capturing || !graph) return fail(ORKAN_EINVAL, "no capture in progress or null output");
  const int fst = flush_pending(h);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  h->capturing = false;
  // nothing ran: the data still has the labels the capture began with
  int end_phys[64];
  std::copy(h->phys, h->phys + 64, end_phys);
  std::copy(h->cap_phys, h->cap_phys + 64, h->phys);
  if (fst != ORKAN_OK) {
    if (g) cudaGraphDestroy(g);
    return fst;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  GraphRec* rec = new (std::nothrow) GraphRec;
  if (!rec) {
    cudaGraphExecDestroy(ex);
    return fail(ORKAN_ENOMEM, "host allocation failed");
  }
  rec->exec = ex;
  rec->n = h->g.n;
  std::copy(h->cap_phys, h->cap_phys + 64, rec->phys_begin);
  std::copy(end_phys, end_phys + 64, rec->phys_end);
  *graph = rec;
  return ORKAN_OK;
}

int orkan_graph_launch(orkan_h h, void* graph) {
  if (int st = check_blocking(h)) return st;
  if (!graph) return fail(ORKAN_EINVAL, "null graph");
  const GraphRec* rec = static_cast<const GraphRec*>(graph);
  // the recorded passes act on physical qubits: the labels must be those the capture began with
  if (rec->n != h->g.n || !std::equal(rec->phys_begin, rec->phys_begin + rec->n, h->phys))
    return fail(ORKAN_EINVAL, "the handle's qubit labels differ from those when the graph was captured");
  if (int st = flush_pending(h)) return st;
  ORKAN_CUDA(cudaGraphLaunch(rec->exec, h->stream));
  std::copy(rec->phys_end, rec->phys_end + 64, h->phys);
  h->n_launches += 1;
  return ORKAN_OK;
}

int orkan_graph_free(void* graph) {
  if (!graph) return ORKAN_OK;
  GraphRec* rec = static_cast<GraphRec*>(graph);
  const cudaError_t e = cudaGraphExecDestroy(rec->exec);
  delete rec;
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphExecDestroy");
  return ORKAN_OK;
}

int orkan_relabel(orkan_h h, const int* phys) {
  if (int st = check_handle(h)) return st;
  if (!phys) return fail(ORKAN_EINVAL, "null map");
  std::vector<char> seen(h->g.n, 0);
  for (int q = 0; q < h->g.n; ++q) {
    if (phys[q] < 0 || phys[q] >= h->g.n || seen[phys[q]]) return fail(ORKAN_EINVAL, "map must be a permutation of 0..n-1");
    seen[phys[q]] = 1;
  }
  int tgt[64];
  for (int q = 0; q < 64; ++q) tgt[q] = q < h->g.n ? phys[q] : q;
  return relabel_to(h, tgt);
}

int orkan_get_labels(orkan_h h, int* phys) {
  if (int st = check_handle(h)) return st;
  if (!phys) return fail(ORKAN_EINVAL, "null output");
  std::copy(h->phys, h->phys + h->g.n, phys);
  return ORKAN_OK;
}

int orkan_set_relabel(orkan_h h, int mode) {
  if (int st = check_handle(h)) return st;
  if (mode != 0 && mode != 1) return fail(ORKAN_EINVAL, "mode must be 0 or 1");
  h->auto_relabel = mode;
  return ORKAN_OK;
}

int orkan_pass_work(orkan_h h, double* alu_ops, double* bytes) {
  if (int st = check_handle(h)) return st;
  if (alu_ops) *alu_ops = h->work_ops;
  if (bytes) *bytes = h->work_bytes;
  h->work_ops = 0.0;
  h->work_bytes = 0.0;
  return ORKAN_OK;
}

int orkan_stats(orkan_h h, int64_t* passes, int64_t* ops, int64_t* launches) {
  if (int st = check_handle(h)) return st;
  if (passes) *passes = h->n_passes;
  if (ops) *ops = h->n_ops;
  if (launches) *launches = h->n_launches;
  return ORKAN_OK;
}

int orkan_set_timing(orkan_h h, int enable) {
  if (int st = check_blocking(h)) return st;
  if (int st = flush_pending(h)) return st;
  h->timing = enable != 0;
  return ORKAN_OK;
}

int orkan_pass_time(orkan_h h, double* ms, int64_t* count) {
  if (int st = check_blocking(h)) return st;
  if (int st = flush_pending(h)) return st;
  ORKAN_CUDA(cudaStreamSynchronize(h->stream));
  double total = 0.0;
  for (auto& p : h->ev_used) {
    float t = 0.0f;
    ORKAN_CUDA(cudaEventElapsedTime(&t, p.first, p.second));
    total += t;
    h->ev_free.push_back(p.first);
    h->ev_free.push_back(p.second);
  }
  if (count) *count = int64_t(h->ev_used.size());
  h->ev_used.clear();
  if (ms) *ms = total;
  return ORKAN_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ autotuner
namespace {

// Fixed probe gates: Rz(a) Ry(b) Rz(c) and CNOT (Ry x Rz), row-major complex128.
void probe_u1(int q, double out[8]) {
  const double a = 0.37 + 0.11 * q, b = 1.1 + 0.07 * q, c = -0.29 + 0.05 * q;
  const cd e1 = std::exp(cd(0, -(a + c) / 2)), e2 = std::exp(cd(0, -(a - c) / 2));
  const cd u00 = e1 * std::cos(b / 2), u01 = -std::conj(e2) * std::sin(b / 2);
  const cd u10 = e2 * std::sin(b / 2), u11 = std::conj(e1) * std::cos(b / 2);
  const cd u[4] = {u00, u01, u10, u11};
  for (int i = 0; i < 4; ++i) { out[2 * i] = u[i].real(); out[2 * i + 1] = u[i].imag(); }
}
void probe_u2(double out[32]) {
  double a[8], b[8];
  probe_u1(1, a);
  probe_u1(2, b);
  Mat A(4), B(4), AB(16), C(16, 0.0);
  for (int i = 0; i < 4; ++i) { A[i] = cd(a[2 * i], a[2 * i + 1]); B[i] = cd(b[2 * i], b[2 * i + 1]); }
  for (int i = 0; i < 4; ++i)   // kron(B, A): bit 0 <-> A
    for (int j = 0; j < 4; ++j) AB[i * 4 + j] = B[(i >> 1) * 2 + (j >> 1)] * A[(i & 1) * 2 + (j & 1)];
  const int perm[4] = {0, 3, 2, 1};   // CNOT, control = index bit 0
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) C[perm[i] * 4 + j] = AB[i * 4 + j];
  for (int i = 0; i < 16; ++i) { out[2 * i] = C[i].real(); out[2 * i + 1] = C[i].imag(); }
}

// One noisy brickwork layer: 1q gate on every qubit, 2q gate on alternating
// neighbour pairs, depolarising on every qubit.
int probe_layer(orkan_h h, int n, int parity) {
  double u1[8], u2[32];
  probe_u2(u2);
  for (int q = 0; q < n; ++q) {
    probe_u1(q, u1);
    if (int st = orkan_apply_unitary(h, 1, &q, u1)) return st;
  }
  for (int q = parity; q + 1 < n; q += 2) {
    const int qs[2] = {q, q + 1};
    if (int st = orkan_apply_unitary(h, 2, qs, u2)) return st;
  }
  for (int q = 0; q < n; ++q)
    if (int st = orkan_depolarize(h, q, 1e-3)) return st;
  return ORKAN_OK;
}

std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int>, std::pair<int, int>> g_tune_cache;

std::string device_name(int dev) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::string s = p.name;
  std::replace(s.begin(), s.end(), ' ', '_');
  return s;
}

}  // namespace

extern "C" int orkan_autotune(int n, int dtype, int* tile_log2, int* max_ops) {
  Geometry g;
  if (!tile_log2 || !max_ops || !valid_dtype(dtype) || !geometry(n, 5, &g))
    return fail(ORKAN_EINVAL, "bad autotune arguments");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(ORKAN_ENODEV, "no CUDA device");
  const auto key = std::make_tuple(dev, n, dtype);
  const std::string gpu = device_name(dev);
  const char* path = std::getenv("ORKAN_TUNE_CACHE");
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *tile_log2 = it->second.first;
      *max_ops = it->second.second;
      return ORKAN_OK;
    }
    if (path) {
      std::ifstream f(path);
      std::string name;
      int fn, fd, fm, ff;
      while (f >> name >> fn >> fd >> fm >> ff) {
        if (name == gpu && fn == n && fd == dtype) {
          g_tune_cache[key] = {fm, ff};
          *tile_log2 = fm;
          *max_ops = ff;
          return ORKAN_OK;
        }
      }
    }
  }
  const int np = std::min(n, 13);
  const int layers = 2;
  float best = 1e30f;
  int best_m = 5, best_f = 8;
  cudaEvent_t e0, e1;
  ORKAN_CUDA(cudaEventCreate(&e0));
  ORKAN_CUDA(cudaEventCreate(&e1));
  for (int m = 3; m <= 5; ++m) {
    for (int f : {1, 2, 4, 8, 16}) {
      orkan_h h = nullptr;
      int st = orkan_alloc(np, dtype, m, &h);
      if (st != ORKAN_OK) continue;
      st = orkan_init_state(h, ORKAN_INIT_MAXMIXED, nullptr);
      if (st == ORKAN_OK) st = orkan_set_fusion(h, f, 1);
      if (st == ORKAN_OK) st = probe_layer(h, np, 0);   // warm-up: kernels loaded, caches set
      if (st == ORKAN_OK) st = orkan_sync(h);
      float ms = 0.0f;
      if (st == ORKAN_OK) {
        cudaEventRecord(e0, h->stream);
        for (int l = 0; l < layers && st == ORKAN_OK; ++l) st = probe_layer(h, np, l & 1);
        if (st == ORKAN_OK) st = orkan_flush(h);
        cudaEventRecord(e1, h->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
          st = ORKAN_ECUDA;
      }
      orkan_free(h);
      if (st != ORKAN_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return st;
      }
      if (ms < best) {
        best = ms;
        best_m = m;
        best_f = f;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = {best_m, best_f};
    if (path) {
      std::ofstream f(path, std::ios::app);
      f << gpu << ' ' << n << ' ' << dtype << ' ' << best_m << ' ' << best_f << '\n';
    }
  }
  *tile_log2 = best_m;
  *max_ops = best_f;
  return ORKAN_OK;
}

// =================================================================== batched circuits
// Host side of orkan_run_batch: every item's ops are prepared in FP64 (Pauli
// transfer matrices for k = 1, qubit-ordered Kraus matrices for k = 2, 3,
// adjoints on observables), packed with the item table, the work slots and
// the readout data into one upload, and run by one persistent launch per
// dtype (batch_kernels.cu).
namespace {

std::mutex g_batch_mutex;          // one batch launch at a time (gangs need their grid resident)
int g_batch_max_ctas = 0;
double g_batch_wait_s = 1.0;

struct BatchArena {
  void* dev = nullptr;
  size_t dev_cap = 0;
  unsigned char* host = nullptr;   // pinned
  size_t host_cap = 0;
};
std::map<int, BatchArena> g_batch_arenas;

int arena_reserve(BatchArena& a, size_t bytes) {
  if (bytes > a.dev_cap) {
    if (a.dev) cudaFree(a.dev);
    a.dev = nullptr;
    a.dev_cap = 0;
    if (cudaMalloc(&a.dev, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(ORKAN_ENOMEM, "batch: device buffer allocation failed");
    }
    a.dev_cap = bytes;
  }
  if (bytes > a.host_cap) {
    if (a.host) cudaFreeHost(a.host);
    a.host = nullptr;
    a.host_cap = 0;
    if (cudaMallocHost(reinterpret_cast<void**>(&a.host), bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(ORKAN_ENOMEM, "batch: pinned host buffer allocation failed");
    }
    a.host_cap = bytes;
  }
  return ORKAN_OK;
}

// Bytes of shared memory a gang-1 item may use for its array.
constexpr size_t kBatchSmemCap = 160 * 1024;

struct PackedBatch {
  std::vector<BatchItem> items;
  std::vector<BatchOp> ops;
  std::vector<double> coef;
  std::vector<unsigned char> aux;
  std::vector<int32_t> slot_item;
  std::vector<int> src;            // item -> index in the caller's array
  std::vector<std::vector<int>> ny;   // per item: Y count of each readout string
  int nres = 0, nmeas = 0;
  int64_t npart = 0;
  size_t smem = 0;
};

size_t aux_put(std::vector<unsigned char>& aux, const void* p, size_t bytes) {
  size_t off = (aux.size() + 15) & ~size_t(15);
  aux.resize(off + bytes);
  std::memcpy(aux.data() + off, p, bytes);
  return off;
}

int batch_fail(int item, int code, const std::string& msg) {
  return fail(code, "batch item " + std::to_string(item) + ": " + msg);
}

// Kraus set of one op in the caller's qubit order (k = 1 channels built here).
int batch_kraus(const orkan_op& o, int item, std::vector<Mat>* out) {
  const int d = 1 << o.k;
  out->clear();
  auto m2 = [](cd a, cd b, cd c, cd dd) { return Mat{a, b, c, dd}; };
  switch (o.kind) {
    case ORKAN_OP_UNITARY:
      if (!o.mats) return batch_fail(item, ORKAN_EINVAL, "null matrix");
      out->push_back(read_mat(o.mats, d));
      return ORKAN_OK;
    case ORKAN_OP_KRAUS:
      if (!o.mats || o.r < 1 || o.r > (1 << (2 * o.k)) || (o.k > 1 && o.r > kK3MaxTerms))
        return batch_fail(item, ORKAN_EINVAL, "need 1 <= r <= min(4^k, 16) Kraus operators");
      for (int t = 0; t < o.r; ++t) out->push_back(read_mat(o.mats + size_t(2) * d * d * t, d));
      return ORKAN_OK;
    case ORKAN_OP_DEPOLARIZE: {
      const double p = o.param;
      if (!(p >= 0.0 && p <= 1.0)) return batch_fail(item, ORKAN_EINVAL, "p must be in [0, 1]");
      const double a = std::sqrt(1.0 - p), b = std::sqrt(p / 3.0);
      *out = {m2(a, 0, 0, a), m2(0, b, b, 0), m2(0, cd(0, -b), cd(0, b), 0), m2(b, 0, 0, -b)};
      return ORKAN_OK;
    }
    case ORKAN_OP_DEPHASE: {
      const double p = o.param;
      if (!(p >= 0.0 && p <= 1.0)) return batch_fail(item, ORKAN_EINVAL, "p must be in [0, 1]");
      const double a = std::sqrt(1.0 - p), b = std::sqrt(p);
      *out = {m2(a, 0, 0, a), m2(b, 0, 0, -b)};
      return ORKAN_OK;
    }
    case ORKAN_OP_AMPDAMP: {
      const double g = o.param;
      if (!(g >= 0.0 && g <= 1.0)) return batch_fail(item, ORKAN_EINVAL, "gamma must be in [0, 1]");
      *out = {m2(1, 0, 0, std::sqrt(1.0 - g)), m2(0, std::sqrt(g), 0, 0)};
      return ORKAN_OK;
    }
  }
  return batch_fail(item, ORKAN_EINVAL, "unknown op kind");
}

// Pauli string (n characters, logical) -> physical masks (x, z, y) and Y count.
int batch_pauli(const char* s, int n, const int* phys, uint64_t m[3], int* ny, int item) {
  m[0] = m[1] = m[2] = 0;
  *ny = 0;
  for (int l = 0; l < n; ++l) {
    const uint64_t bit = uint64_t(1) << phys[l];
    switch (s[l]) {
      case 'I': break;
      case 'X': m[0] |= bit; break;
      case 'Y': m[0] |= bit; m[2] |= bit; ++*ny; break;
      case 'Z': m[1] |= bit; break;
      default: return batch_fail(item, ORKAN_EINVAL, "Pauli characters must be I, X, Y or Z");
    }
  }
  return ORKAN_OK;
}

}  // namespace

namespace {

// Validate item `idx` and append it to the dtype group's tables.
int batch_pack_item(const orkan_batch_item& it, int idx, PackedBatch* pb) {
  orkan_ctx* h = it.h;
  const int n = h->g.n, m = h->g.m, dtype = h->dtype;
  const int64_t N = int64_t(1) << n;
  int phys[64];
  for (int q = 0; q < 64; ++q) phys[q] = q;
  int picture = h->picture;
  if (it.init == ORKAN_BATCH_KEEP) {
    std::copy(h->phys, h->phys + 64, phys);
  } else if (it.init == ORKAN_INIT_PURE) {
    if (!it.init_data) return batch_fail(idx, ORKAN_EINVAL, "ORKAN_INIT_PURE needs init_data");
    picture = ORKAN_STATE;
  } else if (it.init == ORKAN_BATCH_PAULI_SUM) {
    if (it.nterms < 0 || (it.nterms > 0 && (!it.terms || !it.coeffs)))
      return batch_fail(idx, ORKAN_EINVAL, "bad Pauli-sum terms");
    picture = ORKAN_OBSERVABLE;
  } else {
    return batch_fail(idx, ORKAN_EINVAL, "init must be ORKAN_BATCH_KEEP, ORKAN_INIT_PURE or ORKAN_BATCH_PAULI_SUM");
  }
  const bool adj = picture == ORKAN_OBSERVABLE;
  if (it.nops < 0 || (it.nops > 0 && !it.ops)) return batch_fail(idx, ORKAN_EINVAL, "bad op list");
  if (it.npaulis < 0 || (it.npaulis > 0 && (!it.paulis || !it.out)) || (it.psi && !it.out))
    return batch_fail(idx, ORKAN_EINVAL, "readouts need an output array");
  if (it.gang < 0 || it.gang > 64) return batch_fail(idx, ORKAN_EINVAL, "gang must be 0 (automatic) or 1..64");

  BatchItem I{};
  I.state = reinterpret_cast<uint64_t>(h->d_state);
  I.stored = int64_t(h->g.ntiles) << (2 * m);
  I.n = n;
  I.m = m;
  I.psi_off = -1;
  I.op_begin = int32_t(pb->ops.size());
  int nmeas = 0;
  for (int k = 0; k < it.nops; ++k) {
    const orkan_op& o = it.ops[k];
    BatchOp op{};
    if (o.kind == ORKAN_OP_MEASURE || o.kind == ORKAN_OP_PROJECT) {
      if (o.k != 1 && o.k != 0) return batch_fail(idx, ORKAN_EINVAL, "measure / project act on one qubit");
      if (int st = check_qubits_n(n, 1, o.qubits)) return batch_fail(idx, st, g_last_error);
      op.q[0] = phys[o.qubits[0]];
      if (o.kind == ORKAN_OP_MEASURE) {
        if (adj) return batch_fail(idx, ORKAN_EPICTURE, "measurement on an observable (use a projection)");
        if (!(o.param >= 0.0 && o.param < 1.0)) return batch_fail(idx, ORKAN_EINVAL, "u must be in [0, 1)");
        op.form = BF_MEASURE;
        op.u = o.param;
        op.meas = nmeas++;
      } else {
        if (o.outcome != 0 && o.outcome != 1) return batch_fail(idx, ORKAN_EINVAL, "outcome must be 0 or 1");
        op.form = BF_PROJECT;
        op.outcome = o.outcome;
      }
      pb->ops.push_back(op);
      continue;
    }
    const int kq = (o.kind == ORKAN_OP_UNITARY || o.kind == ORKAN_OP_KRAUS) ? o.k : 1;
    if (kq < 1 || kq > 3 || kq > n) return batch_fail(idx, ORKAN_EINVAL, "k must be 1, 2 or 3 and at most n");
    if (int st = check_qubits_n(n, kq, o.qubits)) return batch_fail(idx, st, g_last_error);
    orkan_op oo = o;
    oo.k = kq;
    std::vector<Mat> kraus;
    if (int st = batch_kraus(oo, idx, &kraus)) return st;
    int pq[3];
    for (int l = 0; l < kq; ++l) pq[l] = phys[o.qubits[l]];
    op.coef = int32_t(pb->coef.size());
    if (kq == 1) {
      op.form = BF_PTM1;
      op.q[0] = pq[0];
      const std::vector<double> R = ptm(1, kraus, adj);
      for (int i = 0; i < 16; ++i) {
        double slot;
        pack_slot(dtype, &slot, 0.5 * R[i]);
        pb->coef.push_back(slot);
      }
    } else {
      // bit l of the caller's index is qubit pq[l]; re-index to ascending positions
      int order[3] = {0, 1, 2};
      std::sort(order, order + kq, [&](int x, int y) { return pq[x] < pq[y]; });
      int rank[3] = {0, 0, 0};
      for (int l = 0; l < kq; ++l) {
        op.q[l] = pq[order[l]];
        rank[order[l]] = l;
      }
      const int d = 1 << kq;
      auto perm = [&](int x) {
        int y = 0;
        for (int l = 0; l < kq; ++l) y |= ((x >> l) & 1) << rank[l];
        return y;
      };
      op.form = kq == 2 ? BF_KRAUS2 : BF_KRAUS3;
      op.r = int32_t(kraus.size());
      for (const Mat& K : kraus) {
        Mat B(d * d);
        for (int i = 0; i < d; ++i)
          for (int j = 0; j < d; ++j) B[perm(i) * d + perm(j)] = K[i * d + j];
        if (adj) B = dagger(B, d);   // Phi* applies L^dagger (.) L = M (.) M^dagger with M = L^dagger
        for (int i = 0; i < d * d; ++i) {
          double s0, s1;
          pack_slot(dtype, &s0, B[i].real());
          pack_slot(dtype, &s1, B[i].imag());
          pb->coef.push_back(s0);
          pb->coef.push_back(s1);
        }
      }
    }
    pb->ops.push_back(op);
  }
  I.op_end = int32_t(pb->ops.size());
  I.meas_base = pb->nmeas;
  pb->nmeas += nmeas;
  // initial operator
  if (it.init == ORKAN_INIT_PURE) {
    I.init = 1;
    I.init_off = int64_t(aux_put(pb->aux, it.init_data, size_t(16) * N));
  } else if (it.init == ORKAN_BATCH_PAULI_SUM) {
    I.init = 2;
    I.nterms = it.nterms;
    std::vector<uint64_t> tab(size_t(4) * it.nterms);
    std::vector<double> cs(it.nterms);
    for (int t = 0; t < it.nterms; ++t) {
      uint64_t mk[3];
      int ny = 0;
      if (int st = batch_pauli(it.terms + size_t(t) * n, n, phys, mk, &ny, idx)) return st;
      tab[4 * t] = mk[0];
      tab[4 * t + 1] = mk[1];
      tab[4 * t + 2] = mk[2];
      tab[4 * t + 3] = uint64_t(ny);
      cs[t] = it.coeffs[t];
    }
    std::vector<unsigned char> blob(tab.size() * 8 + cs.size() * 8);
    if (!tab.empty()) std::memcpy(blob.data(), tab.data(), tab.size() * 8);
    if (!cs.empty()) std::memcpy(blob.data() + tab.size() * 8, cs.data(), cs.size() * 8);
    I.init_off = int64_t(aux_put(pb->aux, blob.data(), blob.size()));
  }
  // readouts
  std::vector<int> nys(it.npaulis);
  {
    std::vector<uint64_t> tab(size_t(3) * it.npaulis);
    for (int p = 0; p < it.npaulis; ++p)
      if (int st = batch_pauli(it.paulis + size_t(p) * n, n, phys, &tab[3 * p], &nys[p], idx)) return st;
    I.npauli = it.npaulis;
    I.pauli_off = tab.empty() ? 0 : int64_t(aux_put(pb->aux, tab.data(), tab.size() * 8));
  }
  if (it.psi) {
    std::vector<double> v(size_t(2) * N);
    for (int64_t l = 0; l < N; ++l) {   // logical index l lives at physical index p
      uint64_t p = 0;
      for (int q = 0; q < n; ++q) p |= ((uint64_t(l) >> q) & 1u) << phys[q];
      v[2 * p] = it.psi[2 * l];
      v[2 * p + 1] = it.psi[2 * l + 1];
    }
    I.psi_off = int64_t(aux_put(pb->aux, v.data(), v.size() * 8));
  }
  I.res = pb->nres;
  pb->nres += 2 * it.npaulis + (it.psi ? 1 : 0);
  // gang and placement
  const size_t bytes = h->bytes;
  int G = it.gang;
  // automatic gangs: about 8 Ki stored elements per CTA in native FP64 (GB300's
  // FP64 pipe does 2 operations per SM per clock), 32 Ki on the FP32 pipe
  const int64_t per_cta = dtype == DT_C128 ? 8192 : 32768;
  if (G == 0) G = bytes <= kBatchSmemCap ? 1 : int(std::min<int64_t>(64, std::max<int64_t>(2, (I.stored + per_cta - 1) / per_cta)));
  I.gang = G;
  I.smem = (G == 1 && bytes <= kBatchSmemCap) ? 1 : 0;
  if (I.smem) pb->smem = std::max(pb->smem, (bytes + 15) & ~size_t(15));
  I.part_stride = std::max(2, 2 * it.npaulis + 1);
  I.part_off = pb->npart;
  pb->npart += int64_t(G) * I.part_stride;
  I.first_slot = int32_t(pb->slot_item.size());
  for (int g = 0; g < G; ++g) pb->slot_item.push_back(int32_t(pb->items.size()));
  pb->items.push_back(I);
  pb->src.push_back(idx);
  pb->ny.push_back(nys);
  return ORKAN_OK;
}

}  // namespace

namespace {

// Upload, launch and read back one dtype group; statuses land in items[].status.
int batch_run_group(int dtype, PackedBatch& pb, orkan_batch_item* items, cudaStream_t stream) {
  if (pb.items.empty()) return ORKAN_OK;
  int dev = 0, sms = 0;
  ORKAN_CUDA(cudaGetDevice(&dev));
  ORKAN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int nit = int(pb.items.size());
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  // upload region, then the zeroed region, then the outputs
  size_t off = 0;
  const size_t o_items = off; off = al(off + sizeof(BatchItem) * nit);
  const size_t o_ops = off;   off = al(off + sizeof(BatchOp) * pb.ops.size());
  const size_t o_coef = off;  off = al(off + 8 * pb.coef.size());
  const size_t o_aux = off;   off = al(off + pb.aux.size());
  const size_t o_slot = off;  off = al(off + 4 * pb.slot_item.size());
  const size_t up_bytes = off;
  const size_t o_cnt = off;   off = al(off + 4);
  const size_t o_bar = off;   off = al(off + 4 * size_t(nit));
  const size_t o_stat = off;  off = al(off + 4 * size_t(nit));
  const size_t o_out = off;   off = al(off + 4 * size_t(pb.nmeas));
  const size_t o_prob = off;  off = al(off + 8 * size_t(pb.nmeas));
  const size_t o_res = off;   off = al(off + 8 * size_t(pb.nres));
  const size_t zero_end = off;
  const size_t o_part = off;  off = al(off + 8 * size_t(pb.npart));
  const size_t total = off;
  BatchArena& a = g_batch_arenas[dev];
  if (int st = arena_reserve(a, total)) return st;
  unsigned char* hb = a.host;
  unsigned char* db = static_cast<unsigned char*>(a.dev);
  std::memcpy(hb + o_items, pb.items.data(), sizeof(BatchItem) * nit);
  if (!pb.ops.empty()) std::memcpy(hb + o_ops, pb.ops.data(), sizeof(BatchOp) * pb.ops.size());
  if (!pb.coef.empty()) std::memcpy(hb + o_coef, pb.coef.data(), 8 * pb.coef.size());
  if (!pb.aux.empty()) std::memcpy(hb + o_aux, pb.aux.data(), pb.aux.size());
  std::memcpy(hb + o_slot, pb.slot_item.data(), 4 * pb.slot_item.size());
  BatchDesc d{};
  d.items = reinterpret_cast<const BatchItem*>(db + o_items);
  d.ops = reinterpret_cast<const BatchOp*>(db + o_ops);
  d.coef = reinterpret_cast<const double*>(db + o_coef);
  d.aux = db + o_aux;
  d.slot_item = reinterpret_cast<const int32_t*>(db + o_slot);
  d.counter = reinterpret_cast<int32_t*>(db + o_cnt);
  d.bar = reinterpret_cast<int32_t*>(db + o_bar);
  d.status = reinterpret_cast<int32_t*>(db + o_stat);
  d.outcomes = reinterpret_cast<int32_t*>(db + o_out);
  d.probs = reinterpret_cast<double*>(db + o_prob);
  d.results = reinterpret_cast<double*>(db + o_res);
  d.partials = reinterpret_cast<double*>(db + o_part);
  d.wait_ns = uint64_t(g_batch_wait_s * 1e9);
  d.nslots = int32_t(pb.slot_item.size());
  int per_sm = 0;
  ORKAN_CUDA(batch_occupancy(dtype, pb.smem, &per_sm));
  if (per_sm < 1) return fail(ORKAN_ECUDA, "batch: the kernel does not fit on an SM with this shared memory");
  int grid = std::min<int64_t>(int64_t(per_sm) * sms, d.nslots);
  if (g_batch_max_ctas > 0) grid = std::min(grid, g_batch_max_ctas);
  ORKAN_CUDA(cudaMemcpyAsync(db, hb, up_bytes, cudaMemcpyHostToDevice, stream));
  ORKAN_CUDA(cudaMemsetAsync(db + o_cnt, 0, zero_end - o_cnt, stream));
  ORKAN_CUDA(launch_batch(dtype, d, grid, pb.smem, stream));
  ORKAN_CUDA(cudaMemcpyAsync(hb + o_stat, db + o_stat, zero_end - o_stat, cudaMemcpyDeviceToHost, stream));
  ORKAN_CUDA(cudaStreamSynchronize(stream));
  const int32_t* st = reinterpret_cast<const int32_t*>(hb + o_stat);
  const int32_t* outc = reinterpret_cast<const int32_t*>(hb + o_out);
  const double* prob = reinterpret_cast<const double*>(hb + o_prob);
  const double* res = reinterpret_cast<const double*>(hb + o_res);
  for (int i = 0; i < nit; ++i) {
    const BatchItem& I = pb.items[i];
    orkan_batch_item& it = items[pb.src[i]];
    it.status = st[i];
    int nm = 0;
    for (int k = I.op_begin; k < I.op_end; ++k)
      if (pb.ops[k].form == BF_MEASURE) {
        if (it.outcomes) it.outcomes[nm] = outc[I.meas_base + nm];
        if (it.probs) it.probs[nm] = prob[I.meas_base + nm];
        ++nm;
      }
    for (int p = 0; p < I.npauli; ++p) {
      const double sr = res[I.res + 2 * p], si = res[I.res + 2 * p + 1];
      switch (pb.ny[i][p] & 3) {   // tr(P H) = i^{nY} S
        case 0: it.out[p] = sr; break;
        case 1: it.out[p] = -si; break;
        case 2: it.out[p] = -sr; break;
        default: it.out[p] = si; break;
      }
    }
    if (I.psi_off >= 0) it.out[I.npauli] = res[I.res + 2 * I.npauli];
  }
  return ORKAN_OK;
}

}  // namespace

extern "C" int orkan_batch_limits(int max_ctas, double wait_seconds) {
  if (max_ctas < 0 || !(wait_seconds >= 1e-6 && wait_seconds <= 60.0))
    return fail(ORKAN_EINVAL, "max_ctas must be >= 0 and wait_seconds in [1e-6, 60]");
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  g_batch_max_ctas = max_ctas;
  g_batch_wait_s = wait_seconds;
  return ORKAN_OK;
}

extern "C" int orkan_run_batch(int count, orkan_batch_item* items, void* cuda_stream) {
  if (count < 0 || (count > 0 && !items)) return fail(ORKAN_EINVAL, "bad item list");
  if (count == 0) return ORKAN_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(ORKAN_ENODEV, "no CUDA device");
  for (int i = 0; i < count; ++i) {
    orkan_ctx* h = items[i].h;
    if (int st = check_blocking(h)) return batch_fail(i, st, g_last_error);
    if (h->device != dev) return batch_fail(i, ORKAN_EINVAL, "handle is on another device");
    for (int j = 0; j < i; ++j)
      if (items[j].h == h) return batch_fail(i, ORKAN_EINVAL, "handles must be distinct");
  }
  PackedBatch pb[3];
  for (int i = 0; i < count; ++i) {
    items[i].status = ORKAN_OK;
    if (int st = batch_pack_item(items[i], i, &pb[items[i].h->dtype])) return st;
  }
  // the handles' own work comes first
  for (int i = 0; i < count; ++i) {
    orkan_ctx* h = items[i].h;
    if (int st = flush_pending(h)) return st;
    ORKAN_CUDA(cudaStreamSynchronize(h->stream));
  }
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  {
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    for (int dt = 0; dt < 3; ++dt)
      if (int st = batch_run_group(dt, pb[dt], items, stream)) return st;
  }
  for (int i = 0; i < count; ++i) {
    orkan_ctx* h = items[i].h;
    h->n_launches += 1;
    h->n_ops += items[i].nops;
    if (items[i].init == ORKAN_INIT_PURE || items[i].init == ORKAN_BATCH_PAULI_SUM) {
      reset_labels(h);
      h->picture = items[i].init == ORKAN_INIT_PURE ? ORKAN_STATE : ORKAN_OBSERVABLE;
    }
  }
  for (int i = 0; i < count; ++i)
    if (items[i].status != ORKAN_OK)
      return batch_fail(i, items[i].status, items[i].status == ORKAN_EZEROPROB
                                                ? "a measurement outcome had probability <= 1e-300"
                                                : "the gang barrier's time limit ran out");
  return ORKAN_OK;
}
