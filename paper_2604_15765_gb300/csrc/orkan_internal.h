// Internal definitions shared by the host planner and the CUDA kernels of the
// Orkan GB300 library.  Nothing here is part of the public C ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace orkan {

// Storage / arithmetic policies (public values of orkan_dtype).
enum Dtype : int { DT_C128 = 0, DT_C64 = 1, DT_DF64 = 2 };

// Per-op arithmetic forms.  Every form is applied to a 2^k x 2^k block of the
// operator (Eq. 2, Sec. II-A); the coefficients are prepared on the host in
// FP64 from the Kraus operators.
//   PTM1    : generic single-qubit map, Pauli transfer matrix R/2 (4x4 real)
//   PTM1_U  : unitary single-qubit conjugation, R = 1 (+) R3, coefficients R3/2
//   PTM1_AD : maps that only mix (h00, h11) and scale h01 / h10:
//             h00' = al h00 + be h11, h11' = ga h00 + de h11,
//             h01' = (rho - i sig) h01, h10' = (rho + i sig) h10
//             (depolarising, dephasing, amplitude damping, projectors, Rz)
//   U2      : two-qubit unitary, direct form V h V^dagger (Eq. 2 with r = 1)
//   PTM2    : generic two-qubit map, Pauli transfer matrix R/4 (16x16 real)
//   MONO1 / MONO2 : unitaries whose every row has one non-zero entry, a unit
//             phase i^q (X, Y, Z, S, CNOT, CZ, SWAP, iSWAP, ...): conjugation is
//             a permutation of the block with quarter-turn phase factors,
//             without floating-point arithmetic (Sec. II-B native gates).
//             Coefficients: MONO1 = (p0, p1, q0, q1); MONO2 = the dense V (32
//             slots, for the block form) then (p0..p3, q0..q3).
//   K3 / MONO3 : three-qubit Kraus sets and monomial unitaries; planned on the
//             host like the others but run by their own kernel (K3Desc below),
//             never fused into a pass.
enum OpKind : int {
  OP_PTM1 = 0, OP_PTM1_U = 1, OP_PTM1_AD = 2, OP_U2 = 3, OP_PTM2 = 4, OP_MONO1 = 5, OP_MONO2 = 6,
  OP_K3 = 7, OP_MONO3 = 8
};

constexpr int kMaxOps = 16;     // ops fused into one pass
constexpr int kMaxCoef = 640;   // 8-byte coefficient slots per pass
constexpr int kThreads = 256;   // threads per CTA of the pass kernel

// Slots of an op's coefficients.  Per-part layout (C128, C64, and the
// DF64 forms not listed below): one slot per FP64 coefficient.  DF64 paired
// layout (PTM1, PTM1_U, PTM1_AD): each coefficient use is a lane pair, two
// slots (hi pair, lo pair) -- see pack_op_coefs.
inline int coef_slots(int kind, bool paired = false) {
  switch (kind) {
    case OP_PTM1: return paired ? 32 : 16;
    case OP_PTM1_U: return paired ? 18 : 9;
    case OP_PTM1_AD: return paired ? 14 : 6;
    case OP_U2: return 32;      // 16 complex entries, re/im interleaved
    case OP_PTM2: return 256;
    case OP_MONO1: return 4;
    case OP_MONO2: return 40;
  }
  return 0;
}

struct PassOp {
  int32_t kind;
  int32_t nq;        // 1 or 2
  int32_t rbit[2];   // bit positions in the group row index (ascending)
  int32_t cbit[2];   // bit positions in the group column index (ascending)
  int32_t coef;      // first coefficient slot
  int32_t pad;
};

// One fused pass over the whole tiled operator.  A work item is one tile
// group -- the 2^h x 2^h tiles obtained by inserting every combination of the
// h high-qubit bits into a base tile pair (ti, tj) of the compressed grid, as
// in Algorithm 3 -- restricted to a chunk of 2^rows_log2 rows of each tile.
struct PassDesc {
  int64_t n_items;     // work items: groups * chunks, or ceil(n_tiles / 4) for in-tile passes
  int64_t n_tiles;     // stored tiles
  int32_t has_ptm2;    // 1 if an op of the pass is a generic two-qubit map
  int32_t pad0;
  int64_t nt_c;        // edge of the compressed tile grid (Nt >> h)
  int32_t m;           // tile_log2
  int32_t h;           // number of high (cross-tile) qubits, 0..2
  int32_t hpos[2];     // tile-index bit positions a - m of the high qubits (ascending)
  int32_t rows_log2;   // rows of each tile held per work item
  int32_t chunks_log2; // m - rows_log2
  int32_t nops;
  int32_t skip_diag;   // 1: chunked pass; diagonal groups run in pass_kernel_diag
  PassOp ops[kMaxOps];
  double coef[kMaxCoef];   // F64: double; DF64: float2 (hi, lo) or lane pairs; C64: float in the low half
};

// Three-qubit operations (k = 3): Algorithm 1 on the tiled layout.  One
// launch updates every 8x8 block h_{s,s'} with s >= s' (the others are the
// adjoints of these):
//   form 0 (Kraus sweep): h <- sum_t L_t h L_t^dagger, as the row sweep
//          Y = h L_t^dagger followed by the column sweep L_t Y (Eq. 2);
//          coefficients: per term 64 complex entries of L_t (row-major,
//          re / im in consecutive slots), in the policy's slot format;
//   form 1 (monomial): L[i][p_i] = i^{q_i}, a permutation of the block with
//          quarter-turn phases; slots 0..7 = p, 8..15 = q as raw int64.
// The coefficients travel in the kernel parameter (by value, so a captured
// graph keeps them).
constexpr int kK3MaxTerms = 16;
struct K3Desc {
  int64_t nblocks;   // S (S + 1) / 2 with S = 2^(n - 3)
  int32_t m;         // tile_log2
  int32_t q[3];      // target qubits, ascending
  int32_t form;      // 0 = Kraus sweep, 1 = monomial
  int32_t r;         // Kraus terms of form 0
  double coef[kK3MaxTerms * 128];
};
cudaError_t launch_k3(int dtype, void* state, const K3Desc& d, cudaStream_t stream);

// One op on the packed column-major layout (Sec. III-A), the comparison
// layout: every 2^k x 2^k block h_{s,s'} with s >= s' updated by one thread
// straight from HBM.  Forms: PTM1, PTM1_U, PTM1_AD, MONO1 (k = 1), U2, MONO2
// (k = 2), with the coefficient slots of the pass kernels.
struct PackedDesc {
  int64_t n_blocks;   // S (S + 1) / 2 with S = N / 2^k
  int64_t N;
  int32_t k;
  int32_t kind;
  int32_t q[2];       // ascending
  double coef[40];   // the pass kernels' slots (coef_slots)
};
cudaError_t launch_packed(int dtype, void* state, const PackedDesc& d, cudaStream_t stream);

// Batched circuits (orkan_run_batch): one persistent launch runs the whole
// circuits of many small operators, CTAs taking work slots from a device
// queue; a request runs on `gang` consecutive slots (shared memory when the
// gang is 1 and the array fits).  Op forms:
//   BF_PTM1   : k = 1, coefficients R / 2 (4 x 4 real Pauli transfer matrix)
//   BF_KRAUS2 : k = 2, r terms of 16 complex entries (row-major, re / im slots)
//   BF_KRAUS3 : k = 3, r terms of 64 complex entries
//   BF_MEASURE: Z measurement of q[0] with draw u, Born renormalisation
//   BF_PROJECT: Pi_outcome (.) Pi_outcome, no renormalisation
constexpr int kBatchThreads = 256;
enum BatchForm : int32_t { BF_PTM1 = 0, BF_KRAUS2 = 1, BF_KRAUS3 = 2, BF_MEASURE = 3, BF_PROJECT = 4 };
struct BatchOp {
  int32_t form;
  int32_t r;         // Kraus terms
  int32_t q[3];      // physical qubits, ascending
  int32_t coef;      // first 8-byte coefficient slot
  int32_t meas;      // BF_MEASURE: index of its outcome / probability within the request
  int32_t outcome;   // BF_PROJECT
  double u;          // BF_MEASURE: uniform draw
};
struct BatchItem {
  uint64_t state;      // device address of the tiled array
  int64_t stored;      // stored elements
  int64_t init_off;    // aux byte offset of the initial data (init 1: N complex; init 2: term table)
  int64_t pauli_off;   // aux byte offset of the readout strings (3 uint64 masks x, z, y each)
  int64_t psi_off;     // aux byte offset of the readout vector (N complex), or -1
  int64_t part_off;    // first double of the gang's scratch partial sums
  int32_t n, m;
  int32_t init;        // 0: the array as it is, 1: pure state, 2: Pauli sum
  int32_t nterms;      // init 2
  int32_t op_begin, op_end;
  int32_t npauli;
  int32_t res;         // first result slot (2 per string, then <psi|H|psi>)
  int32_t meas_base;   // first outcome / probability slot
  int32_t gang;        // CTAs working on the request
  int32_t first_slot;  // its first work slot
  int32_t smem;        // 1: staged in shared memory (gang 1)
  int32_t part_stride; // doubles of scratch per gang member
  int32_t pad;
};
struct BatchDesc {
  const BatchItem* items;
  const BatchOp* ops;
  const double* coef;
  const unsigned char* aux;
  const int32_t* slot_item;  // work slot -> request
  int32_t* counter;          // queue head (zero at launch)
  int32_t* bar;              // per request: barrier arrivals (zero at launch)
  int32_t* status;           // per request: ORKAN_OK, ORKAN_EZEROPROB or ORKAN_ETIMEOUT (zero at launch)
  double* partials;
  double* results;
  int32_t* outcomes;
  double* probs;
  uint64_t wait_ns;          // time limit of one gang barrier
  int32_t nslots;
  int32_t pad;
};
cudaError_t launch_batch(int dtype, const BatchDesc& d, int grid, size_t smem, cudaStream_t stream);
cudaError_t batch_occupancy(int dtype, size_t smem, int* per_sm);

// Tensor-core pass (tc_kernels.cu): every stored tile T <- L T L^dagger for one
// composed in-tile unitary L (m = 5, 32 x 32, complex64 storage), on tcgen05
// MMAs.  u: L row-major as (re, im) floats; err: device word set to 1 if a
// bounded wait ran out.  The matrix travels in the kernel parameter.
struct TcDesc {
  int64_t ntiles;
  int32_t* err;
  float2 u[32 * 32];
};
cudaError_t launch_tc(void* state, const TcDesc& d, cudaStream_t stream);

// Record the message that orkan_last_error() returns on the calling thread.
void set_last_error(const char* msg);

// Launchers (pass_kernels.cu).  Return cudaSuccess or the launch error;
// *launches receives the number of kernels launched (1 or 2).
cudaError_t launch_pass(int dtype, void* state, const PassDesc& d, cudaStream_t s, int* launches);

// Auxiliary kernels (aux_kernels.cu).
struct Geometry {
  int n;
  int m;
  int64_t N;       // 2^n
  int64_t Nt;      // tile rows (>= 1)
  int64_t ntiles;  // Nt (Nt + 1) / 2
};
cudaError_t launch_zero(int dtype, void* state, const Geometry& g, cudaStream_t s);
// Tiled <-> packed column-major copies of one operator (to_packed = 1: tiled -> packed).
cudaError_t launch_packed_convert(int dtype, void* packed, void* tiled, const Geometry& g, int to_packed,
                                  cudaStream_t stream);
cudaError_t launch_set_diag(int dtype, void* state, const Geometry& g, int64_t i, double re, cudaStream_t s);
cudaError_t launch_fill_diag(int dtype, void* state, const Geometry& g, double re, cudaStream_t s);
cudaError_t launch_from_dense(int dtype, void* state, const Geometry& g, const double* dense_dev, cudaStream_t s);
cudaError_t launch_from_pure(int dtype, void* state, const Geometry& g, const double* psi_dev, cudaStream_t s);
cudaError_t launch_to_dense(int dtype, const void* state, const Geometry& g, double* dense_dev, cudaStream_t s);
cudaError_t launch_gather(int dtype, const void* state, const Geometry& g, int64_t count, const int64_t* rows_dev,
                          const int64_t* cols_dev, double* out_dev, cudaStream_t s);
cudaError_t launch_pauli_sum(int dtype, void* state, const Geometry& g, int nterms, const uint64_t* masks_dev,
                             const double* coeffs_dev, cudaStream_t s);
// Reductions write into a device double[4] result (after a fixed-order two-stage reduction).
//   diag:  res = {sum Re h_ii, sum Im h_ii, sum_{bit q of i = 0} Re h_ii, sum_{bit q = 1} Re h_ii}
//   pauli: res = {Re S, Im S} with S = sum_i sign(i) h[i ^ x, i]
//   expect: res = {sum_tiles w Re <O_t, rho_t>_F}
constexpr int kRedBlocks = 608;   // 4 x 152 SMs; fixed so the summation order is fixed
cudaError_t launch_reduce_diag(int dtype, const void* state, const Geometry& g, int q, double* partials,
                               double* res, cudaStream_t s);
cudaError_t launch_reduce_pauli(int dtype, const void* state, const Geometry& g, uint64_t xmask, uint64_t zmask,
                                uint64_t ymask, double* partials, double* res, cudaStream_t s);
cudaError_t launch_reduce_expect(int dtype, const void* rho, const void* O, const Geometry& g, double* partials,
                                 double* res, cudaStream_t s);

}  // namespace orkan
