/*
 * orkan.h -- C ABI of the Orkan GB300 library: single-pass k-local conjugation
 * of a hermitian operator stored in the tiled lower-triangle layout.
 *
 * The method (arXiv:2604.15765, "Orkan: Cache-friendly simulation of quantum
 * operations on hermitian operators"):
 *   - Eq. (1), Sec. II: a quantum operation in Kraus form,
 *       Phi(H) = sum_alpha K_alpha H K_alpha^dagger,
 *     acting on any hermitian H (a density matrix or an observable).
 *   - Sec. I / Sec. II: the Heisenberg picture applies the trace-dual map
 *       Phi*(O) = sum_alpha K_alpha^dagger O K_alpha.
 *   - Sec. II-A, Eq. (2), Algorithm 1: a k-local operation K = I (x) L
 *     updates every 2^k x 2^k block h_{s,s'} independently:
 *     h -> sum L h L^dagger (k = 1, 2, 3 here).
 *   - Sec. III-A: the packed column-major lower triangle, kept as the
 *     comparison layout (orkan_packed_*).
 *   - Sec. III-B: storage keeps the lower triangle at tile granularity
 *     (tiles of edge M = 2^m, tile (ti, tj) with ti >= tj, tiles row-major,
 *     elements row-major in a tile, diagonal tiles complete, zero padding to
 *     one M x M tile if N < M).  N (N + M) / 2 elements (Table I).
 *   - Sec. III-C: the mean value tr(rho O) as per-tile Frobenius products.
 *
 * Conventions
 *   - Qubit a is bit a of a basis index (qubit 0 = least significant bit).
 *   - A 2^k x 2^k matrix L given with qubits[0..k-1] maps bit l of its own
 *     row/column index to qubit qubits[l].  Matrices are row-major,
 *     complex128 interleaved (re, im), i.e. 2 * 4^k doubles.
 *   - Handles are stream-ordered: every call enqueues work on the handle's
 *     CUDA stream and returns; calls that return scalars or host data wait
 *     for the stream.  Consecutive operations are fused into one pass over
 *     the state when their qubits allow it (see orkan_set_fusion).
 *   - Input matrices and strings are copied during the call; the caller
 *     keeps ownership of every pointer it passes.
 *   - A handle is used from one host thread at a time.
 *
 * Status codes: ORKAN_OK (0) or a negative ORKAN_E* value; no C++ exception
 * ever crosses this boundary.  orkan_strerror() names a code and
 * orkan_last_error() returns a message for the calling thread's last error.
 */
#ifndef ORKAN_H
#define ORKAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORKAN_OK 0
#define ORKAN_EINVAL (-1)    /* bad argument: qubit out of range or repeated, k > 3, r > 4^k, ... */
#define ORKAN_ENOMEM (-2)    /* device or host allocation failed */
#define ORKAN_ECUDA (-3)     /* a CUDA call failed (message in orkan_last_error) */
#define ORKAN_EZEROPROB (-4) /* measurement: the selected outcome has probability < 1e-300 */
#define ORKAN_EPICTURE (-5)  /* operation not defined in the handle's picture */
#define ORKAN_ENODEV (-6)    /* no CUDA device */
#define ORKAN_ETIMEOUT (-7)  /* a bounded device-side wait ran out (orkan_run_batch gang barrier) */

/* Storage dtype.
 *   ORKAN_C128: complex128 elements, native FP64 arithmetic (16 B/element).
 *   ORKAN_C64 : complex64 elements, FP32 arithmetic (8 B/element).
 *   ORKAN_DF64: "double-float" elements -- real and imaginary part each kept
 *               as an unevaluated sum hi + lo of two floats (16 B/element,
 *               stored as the floats re.hi, im.hi, re.lo, im.lo) -- with
 *               FP32-pipe error-free arithmetic, about 48 significand bits.
 *               Values must stay within the float exponent range
 *               (|x| < 3e38; parts below 1e-38 flush to zero).
 * Readouts (trace, probabilities, expectations) accumulate in FP64 for all. */
#define ORKAN_C128 0
#define ORKAN_C64 1
#define ORKAN_DF64 2

/* Picture of a handle, set by orkan_init_state / orkan_init_observable. */
#define ORKAN_STATE 0
#define ORKAN_OBSERVABLE 1

/* orkan_init_state kinds. */
#define ORKAN_INIT_ZERO 0     /* |0...0><0...0|, data ignored */
#define ORKAN_INIT_MAXMIXED 1 /* I / N, data ignored */
#define ORKAN_INIT_DENSE 2    /* data: N x N complex128 row-major (2 N^2 doubles); lower triangle is read */
#define ORKAN_INIT_PURE 3     /* data: N complex128 amplitudes psi (2 N doubles); rho = psi psi^dagger */

typedef struct orkan_ctx *orkan_h;

/* ------------------------------------------------------------------ errors */
const char *orkan_strerror(int status);
/* Message of the calling thread's most recent failing call ("" if none). */
const char *orkan_last_error(void);

/* ------------------------------------------------------------------ layout (host only, no GPU needed)
 * Sec. III-B and Table I. */

/* Bytes of the tiled array: N (N + M) / 2 elements, or M^2 if N < M, times the
 * element size (16 for C128 and DF64, 8 for C64).  0 on bad arguments. */
size_t orkan_bytes(int n, int dtype, int tile_log2);

/* Number of stored tiles Nt (Nt + 1) / 2 with Nt = max(1, N / M); -1 on bad arguments. */
int64_t orkan_num_tiles(int n, int tile_log2);

/* Element offset of H[i, j] in the tiled array; *conj is set to 1 when the
 * stored value is the conjugate of H[i, j] (i < j), else 0.  -1 if out of range. */
int64_t orkan_element_offset(int n, int tile_log2, int64_t i, int64_t j, int *conj);

/* Subroutine 1 (insertBits): the global index whose bits at the ascending
 * positions pos[0..k-1] are the bits of a (bit l at pos[l]) and whose other
 * bits, in order, are the bits of s. */
uint64_t orkan_insert_bits(uint64_t s, uint64_t a, int k, const int *pos);

/* Pauli transfer matrix of the k-local map with r Kraus operators K (r
 * matrices of 2^k x 2^k, layout as above), in FP64 on the host:
 *   R[a][b] = 2^-k tr(P_a Phi(P_b)), P_a = sigma_{a_{k-1}} (x) ... (x) sigma_{a_0},
 * a = a_0 + 4 a_1 (sigma_0..3 = I, X, Y, Z).  adjoint != 0 gives the map
 * Phi* instead.  out: 16^k doubles, row-major.  This is the representation
 * the kernels apply for single-qubit maps (the transfer matrix of Eq. (3) in
 * the Pauli basis, where it is real). */
int orkan_ptm(int k, int r, const double *K, int adjoint, double *out);

/* ------------------------------------------------------------------ lifetime */

/* Storage of Sec. III-B (tiled lower triangle, Table I footprint).
 * Allocate an n-qubit operator (1 <= n <= 24) with tile edge 2^tile_log2
 * (3 <= tile_log2 <= 5; the paper's m = 5 is the default when tile_log2 is 0)
 * on the current CUDA device.  The content is undefined until an init call.
 * Errors: EINVAL, ENOMEM, ENODEV, ECUDA. */
int orkan_alloc(int n, int dtype, int tile_log2, orkan_h *out);

/* Same, on caller-owned device memory of at least orkan_bytes(...) bytes,
 * 256-byte aligned (e.g. a torch tensor); orkan_free does not release it. */
int orkan_alloc_external(int n, int dtype, int tile_log2, void *dev_ptr, size_t bytes, orkan_h *out);

/* Sec. III-B storage lifetime.
 * Wait for the handle's work and release it (and its memory unless external). */
int orkan_free(orkan_h h);

/* Run the handle's work on the given cudaStream_t (NULL = the legacy default
 * stream).  Pending fused ops are flushed on the old stream first. */
int orkan_set_stream(orkan_h h, void *cuda_stream);

/* Fusion policy: at most max_ops (1..16) consecutive ops per pass; compose
 * != 0 lets consecutive single-qubit ops on the same qubit be multiplied
 * into one transfer matrix in FP64 on the host, and (with max_ops >= 2) holds
 * single-Kraus single-qubit ops back per qubit so that the next dense
 * two-qubit single-Kraus op on that qubit absorbs them (one 4 x 4 product in
 * FP64); any other op on the qubit, the end of an orkan_run_circuit call and
 * every flush or blocking call release them first.  Default: 8, 1.
 * max_ops = 1 with compose = 0 is the plain one-pass-per-op path. */
int orkan_set_fusion(orkan_h h, int max_ops, int compose);

/* Tensor-core passes for in-tile runs (complex64 handles with tile_log2 = 5;
 * no counterpart in the paper, which applies ops one by one).  A run of
 * consecutive single-Kraus ops (unitaries, or one-operator Kraus sets) on
 * qubits below the tile size is, as a whole, one operator L_blk on the tile's
 * 5 qubits (composed in FP64 on the host); it maps every stored tile T to
 * L_blk T L_blk^dagger (Eq. 2 with k = m, Sec. III-C intra-tile case), two
 * dense complex 32 x 32 x 32 products per tile whatever the run's length,
 * run on tcgen05 tensor cores with split-TF32 operands (about 2^-22 relative
 * per pass; complex64 storage holds 2^-24).  Such a run then holds up to 64
 * ops instead of the fusion depth.  mode 0: off (the default of C128 and
 * DF64 handles, which it does not serve); 1: runs with at least two dense
 * two-qubit ops or at least six ops (the default of C64 handles); 2: every
 * such run.  An in-tile three-qubit single-Kraus op joins such a run (it then
 * always runs as a tensor-core pass).  A fusion depth of 1 (orkan_set_fusion)
 * keeps the plain one-pass-per-op path whatever the mode.  Other handles and
 * ops are unaffected.  A bounded wait inside the pass that runs out makes the
 * next orkan_sync return ORKAN_ETIMEOUT (the operator is then undefined).
 * Errors: EINVAL. */
int orkan_set_tensor(orkan_h h, int mode);

int orkan_get_info(orkan_h h, int *n, int *dtype, int *tile_log2, int *picture);

/* Autotuner: the tile size (tile_log2, 3..5) and fusion depth (max_ops,
 * 1..16, with composition) that run a noisy brickwork probe fastest on the
 * current device for n-qubit operators of dtype.  It times one warm-up and two
 * probe layers (a 1-qubit gate on every qubit, 2-qubit gates on alternating
 * neighbour pairs, depolarising on every qubit) on min(n, 13) qubits for every
 * candidate pair, allocating and freeing temporary operators.  The choice is
 * cached per (device, n, dtype) for the process and, when the environment
 * variable ORKAN_TUNE_CACHE names a file, read from / appended to it.
 * Errors: EINVAL, ENODEV, ENOMEM, ECUDA.  (Not in the paper, which fixes m = 5.) */
int orkan_autotune(int n, int dtype, int *tile_log2, int *max_ops);

/* Device address of the tiled array (layout of Sec. III-B, element type of the
 * dtype), indexed by physical qubit labels (the identity unless orkan_relabel
 * or the automatic planner moved qubits; see orkan_get_labels). */
void *orkan_device_ptr(orkan_h h);

/* ------------------------------------------------------------------ initialisation */

/* Sec. III-B layout, Sec. II (a state is the hermitian H that Phi acts on).
 * Set the handle to a state (picture ORKAN_STATE).  See ORKAN_INIT_*.
 * Errors: EINVAL (unknown kind, NULL data for DENSE/PURE), ENOMEM, ECUDA. */
int orkan_init_state(orkan_h h, int kind, const double *data);

/* Sec. I / Sec. II trace duality: the observable is the operand of the
 * Heisenberg picture.  Set the handle to the observable O = sum_t coeffs[t] P_t (picture
 * ORKAN_OBSERVABLE).  paulis: nterms strings of n characters from "IXYZ"
 * back to back (no separators); character l acts on qubit l.
 * Errors: EINVAL (bad character, nterms < 0), ENOMEM, ECUDA. */
int orkan_init_observable(orkan_h h, int nterms, const char *paulis, const double *coeffs);

/* Declare the handle's operator a state (Phi applies) or an observable (Phi*
 * applies), e.g. after loading an observable with ORKAN_INIT_DENSE.  Pending
 * ops are flushed in the old picture first. */
int orkan_set_picture(orkan_h h, int picture);

/* Raw tiled array copies (checkpoint / resume): host_src / host_dst hold
 * orkan_bytes(...) bytes in the handle's dtype and layout. */
int orkan_load_tiled(orkan_h h, const void *host_src, int picture);
int orkan_store_tiled(orkan_h h, void *host_dst);

/* Checkpoints (not in the paper): a header of ORKAN_CKPT_HEADER_BYTES bytes
 * followed by the raw tiled array (Sec. III-B layout) as the handle holds
 * it, in physical qubit order, so saving needs no relabelling pass.  Header,
 * little-endian: 8 bytes magic "ORKANCK1"; int32 version (1), n, tile_log2,
 * dtype, picture, 0; int32 phys[64] (physical position of logical qubit q,
 * q < n; entries from n on are q); uint64 data bytes (= orkan_bytes(n,
 * dtype, tile_log2)); uint64 checksum of the data (FNV-1a over 64-bit
 * little-endian words: h = 0xcbf29ce484222325, h = (h ^ w) * 0x100000001b3);
 * zero padding to ORKAN_CKPT_HEADER_BYTES.  Host buffers are the caller's.
 *   orkan_checkpoint_bytes: bytes a checkpoint of h takes (0 for NULL).
 *   orkan_checkpoint_save: flush h's pending ops and write its checkpoint to
 *     host_dst (cap bytes; EINVAL if smaller than orkan_checkpoint_bytes).
 *   orkan_checkpoint_load: check the header (magic, version, sizes, labels,
 *     checksum) and that n, tile_log2 and dtype equal h's, then load the data,
 *     the picture and the labels into h.  A mismatch is EINVAL with both
 *     shapes named, and leaves h unchanged.
 *   orkan_checkpoint_inspect: host only (no GPU), the same checks and the
 *     header's n, dtype, tile_log2 and picture (any output may be NULL). */
#define ORKAN_CKPT_HEADER_BYTES 320
size_t orkan_checkpoint_bytes(orkan_h h);
int orkan_checkpoint_save(orkan_h h, void *host_dst, size_t cap);
int orkan_checkpoint_load(orkan_h h, const void *host_src, size_t bytes);
int orkan_checkpoint_inspect(const void *host_src, size_t bytes, int *n, int *dtype, int *tile_log2, int *picture);

/* orkan_load_tiled without the wait: the copy is queued on the handle's
 * stream and the call returns.  Later calls on h are ordered after the copy;
 * host_src must stay valid and unchanged until it has completed (after
 * orkan_sync(h) or any blocking call on h).  From pinned host memory the copy
 * runs asynchronously, so an upload to one handle can overlap the passes of
 * a handle on another stream; from pageable memory the driver may finish it
 * before returning.  Host-device plumbing with no counterpart in the paper.
 * Errors: EINVAL (NULL host_src, bad picture, during graph capture), ECUDA. */
int orkan_load_tiled_async(orkan_h h, const void *host_src, int picture);

/* ------------------------------------------------------------------ operations
 * On a STATE handle these apply Phi (Eq. 1); on an OBSERVABLE handle Phi*
 * (the caller issues a circuit's ops in reverse order for Heisenberg
 * evolution). */

/* Unitary gate U (2^k x 2^k, k = 1, 2 or 3) on qubits[0..k-1] (distinct, < n).
 * k = 1, 2: fused into passes over tile groups (Sec. III-C).  k = 3: the
 * block update of Algorithm 1 (Sec. II-A) in its own launch, every 8x8 block
 * h_{s,s'} with s >= s' gathered from the tiled layout (up to 64 tiles per
 * block, Sec. III-C); monomial U (Toffoli, CCZ, Fredkin, ...) permute the
 * block without arithmetic. */
int orkan_apply_unitary(orkan_h h, int k, const int *qubits, const double *U);

/* Kraus map with r (1 <= r <= 4^k) operators K (r matrices back to back) on
 * k = 1, 2 or 3 qubits; for k = 3 at most 16 operators (EINVAL above).  Trace
 * non-increase is not checked. */
int orkan_apply_kraus(orkan_h h, int k, const int *qubits, int r, const double *K);

/* Depolarising channel of Sec. IV-A: Kraus sqrt(1-p) I, sqrt(p/3) {X, Y, Z}. */
int orkan_depolarize(orkan_h h, int q, double p);
/* Dephasing (phase flip): sqrt(1-p) I, sqrt(p) Z.  Not defined in the paper. */
int orkan_dephase(orkan_h h, int q, double p);
/* Amplitude damping: diag(1, sqrt(1-gamma)), sqrt(gamma)|0><1|.  Not defined in the paper. */
int orkan_amplitude_damp(orkan_h h, int q, double gamma);

/* Sec. II: the projectors Pi_0, Pi_1 form a CP trace non-increasing map;
 * Born renormalisation is not in the paper (it mentions only trace
 * non-increasing maps), so the reading here is p_b = tr(Pi_b rho) and
 * rho <- Pi_b rho Pi_b / p_b.
 * Z-basis measurement of qubit q on a STATE handle with the caller's uniform
 * draw u in [0, 1): p_b = tr(Pi_b rho) in FP64, outcome = 0 iff
 * u (p0 + p1) < p0, then rho <- Pi_b rho Pi_b / p_b (Born renormalisation).
 * *outcome and *prob (= p_b / (p0 + p1)) are written on success.
 * Blocks until the probabilities are known.
 * Errors: EPICTURE on an observable, EZEROPROB, EINVAL. */
int orkan_measure(orkan_h h, int q, double u, int *outcome, double *prob);

/* Sec. II (CP trace non-increasing map with the single Kraus operator
 * Pi_b, self-adjoint): Pi_b H Pi_b without renormalisation (both pictures). */
int orkan_project(orkan_h h, int q, int outcome);

/* ------------------------------------------------------------------ whole circuits in one call */
#define ORKAN_OP_UNITARY 0    /* mats: one 2^k x 2^k matrix */
#define ORKAN_OP_KRAUS 1      /* mats: r matrices */
#define ORKAN_OP_DEPOLARIZE 2 /* param = p */
#define ORKAN_OP_DEPHASE 3    /* param = p */
#define ORKAN_OP_AMPDAMP 4    /* param = gamma */
#define ORKAN_OP_MEASURE 5    /* param = u (state handles only) */
#define ORKAN_OP_PROJECT 6    /* outcome */

typedef struct {
  int kind;           /* ORKAN_OP_* */
  int k;              /* qubits acted on (1 to 3; 1 for channels, measure, project) */
  int qubits[3];
  int r;              /* Kraus operators (ORKAN_OP_KRAUS) */
  int outcome;        /* ORKAN_OP_PROJECT */
  double param;       /* p, gamma or the uniform draw u */
  const double *mats; /* complex128 matrices, row-major interleaved (UNITARY, KRAUS) */
} orkan_op;

/* Apply ops[0..count-1] in order with exactly the semantics of the single
 * calls (orkan_apply_unitary, ..., orkan_measure, orkan_project); the j-th
 * MEASURE op writes outcomes[j] and probs[j] (either may be NULL).  Stops at
 * the first failing op and returns its status; *done (if not NULL) receives
 * the number of ops applied.  One call per circuit keeps host overhead per op
 * in the microseconds. */
int orkan_run_circuit(orkan_h h, int count, const orkan_op *ops, int *outcomes, double *probs, int *done);

/* ------------------------------------------------------------------ batched circuits
 * Many small operators' whole circuits in one persistent launch per dtype:
 * Eq. (1) / Eq. (2) block updates of Algorithm 1 on each tiled array
 * (Sec. III-B), Z projections with Born renormalisation (Sec. II trace
 * non-increasing maps, renormalised as orkan_measure does), then the
 * readouts tr(P H) (Pauli strings) and <psi|H|psi> (Sec. III-C mean value
 * against a pure state).  For operators whose per-op passes are too short
 * to fill the GPU (n up to ~10): CTAs take work slots from a device queue;
 * an operator that fits shared memory (n <= 7) runs its whole circuit in one
 * CTA with one read and one write of its array, a larger one on a gang of
 * CTAs that meet at a time-limited barrier between ops.  Results depend only
 * on the item itself (fixed reduction orders), never on the rest of the
 * batch.
 *
 * Per item:
 *   h       the operator's handle (its n, dtype, tile size and memory); its
 *           pending ops are flushed and its stream waited for first.
 *   init    ORKAN_BATCH_KEEP: h's current operator, picture and labels;
 *           ORKAN_INIT_PURE: rho = psi psi^dagger from init_data (N complex,
 *           2 N doubles), picture STATE, labels reset;
 *           ORKAN_BATCH_PAULI_SUM: O = sum_t coeffs[t] P_t from nterms strings
 *           `terms` (nterms * n characters of IXYZ, character l on qubit l),
 *           picture OBSERVABLE, labels reset.
 *   nops, ops  the circuit, with orkan_run_circuit's op semantics (MEASURE
 *           only on states; on an observable every op applies Phi*).
 *           k = 1 maps run as their Pauli transfer matrix, k = 2, 3 as Kraus
 *           sweeps (at most 16 operators).  No fusion or composition.
 *   npaulis, paulis  readout strings (npaulis * n characters), logical qubits.
 *   psi     readout vector (N complex, logical index order) or NULL.
 *   out     host: npaulis values tr(P H), then <psi|H|psi> if psi.
 *   outcomes, probs  host, one per MEASURE op (either may be NULL).
 *   gang    0: automatic (1 when the array fits shared memory, else about
 *           one CTA per 8 Ki (C128) or 32 Ki (C64, DF64) stored elements, at
 *           most 64); else the number of CTAs to use (1..64).
 *   status  written by the call: ORKAN_OK, ORKAN_EZEROPROB (a measurement
 *           outcome had probability <= 1e-300; the item stopped there) or
 *           ORKAN_ETIMEOUT (its gang did not assemble within the wait limit,
 *           e.g. a gang larger than the grid; the item stopped there).
 * The call validates every item before launching (EINVAL / EPICTURE name
 * the item), blocks until the results are on the host and returns ORKAN_OK
 * when every item succeeded, else the first failing item's status.  Work
 * runs on cuda_stream (NULL = the legacy default stream).  Handles must be
 * distinct and on the current device.  Calls from several host threads are
 * serialised per device (a gang needs every CTA of its launch resident). */
#define ORKAN_BATCH_KEEP (-1)
#define ORKAN_BATCH_PAULI_SUM 4
typedef struct {
  orkan_h h;
  int init;
  const double *init_data;
  int nterms;
  const char *terms;
  const double *coeffs;
  int nops;
  const orkan_op *ops;
  int npaulis;
  const char *paulis;
  const double *psi;
  double *out;
  int *outcomes;
  double *probs;
  int gang;
  int status;
} orkan_batch_item;
int orkan_run_batch(int count, orkan_batch_item *items, void *cuda_stream);

/* Process-wide limits of orkan_run_batch: at most max_ctas CTAs per launch
 * (0 = as many as can be resident, which is also the upper bound), and the
 * time limit of one gang barrier in seconds (default 1.0; 1e-6 .. 60). */
int orkan_batch_limits(int max_ctas, double wait_seconds);

/* ------------------------------------------------------------------ readouts (block; FP64) */

/* Sec. III-C (the diagonal of the diagonal tiles): tr H = sum_i H_ii (re, im). */
int orkan_trace(orkan_h h, double *re, double *im);

/* Sec. I / Sec. III-C mean value tr(rho O) with O a Pauli string: tr(P H)
 * for P given as n characters of "IXYZ", character l on (logical) qubit l;
 * reads the N elements H[i ^ x, i] (x = the string's X/Y mask). */
int orkan_expect_pauli(orkan_h h, const char *pauli, double *out);

/* tr(rho O) as tiled Frobenius products (Sec. III-C; diagonal tiles once,
 * strictly lower tiles twice).  Both handles: same n, tile size and dtype. */
int orkan_expect(orkan_h rho, orkan_h O, double *out);

/* Sec. III-B (the inverse of the tiled map, upper tiles mirrored from the
 * stored lower ones).
 * Dense N x N complex128 row-major copy into host memory out (2 N^2 doubles).
 * Elements above the diagonal are conjugates of the stored lower ones. */
int orkan_to_dense(orkan_h h, double *out);

/* Gather count elements H[rows[t], cols[t]] (any triangle; upper ones are
 * conjugated stored values) into host memory out (2 count doubles, complex128).
 * rows / cols: host arrays of count indices in [0, N).  Errors: EINVAL. */
int orkan_get_elements(orkan_h h, int64_t count, const int64_t *rows, const int64_t *cols, double *out);

/* Launch any pending fused ops / wait for the handle's stream. */
int orkan_flush(orkan_h h);
int orkan_sync(orkan_h h);

/* ------------------------------------------------------------------ captured circuits
 * Record the passes that the operations applied to h launch (a circuit of
 * unitaries, channels and projections; fusion applies) into an executable
 * CUDA graph, and replay it on the same handle: each replay applies the
 * circuit again to the handle's current operator, without host planning or
 * per-op launches.  Recording does not execute the circuit.  Between begin and
 * end only operation calls are allowed; blocking calls (measure, readouts,
 * init, sync) fail with EINVAL.  The handle needs a non-default stream (its
 * own, or one set with orkan_set_stream).  A graph is bound to the handle's
 * device memory and stays valid until orkan_graph_free.  It replays physical
 * passes: recording leaves the labels as they were at orkan_capture_begin;
 * launching needs those labels (EINVAL otherwise) and leaves the labels the
 * recorded calls ended with. */
int orkan_capture_begin(orkan_h h);
int orkan_capture_end(orkan_h h, void **graph);
int orkan_graph_launch(orkan_h h, void *graph);
int orkan_graph_free(void *graph);

/* ------------------------------------------------------------------ qubit relabelling
 * A handle keeps a map from logical qubits (the numbers every call takes and
 * returns) to physical bit positions of the tiled layout, the identity after
 * allocation and every init / load.  Relabelling moves data so that qubits a
 * circuit uses often sit below the tile size m, where their ops run inside
 * tiles and fuse freely, instead of spanning tile groups (Sec. III-C).  The
 * operator a handle represents never changes: operations, measurements,
 * Pauli expectations, elements and dense exports all translate through the
 * map; orkan_expect relabels O to rho's map first; orkan_store_tiled and
 * orkan_packed_from_tiled restore the identity map first (passes).  The
 * allocation-free readout reads the physical layout as it is. */

/* Set the map: phys[q] = physical position of logical qubit q (a permutation
 * of 0..n-1).  Applied as at most n - 1 SWAP permutation passes (fused). */
int orkan_relabel(orkan_h h, const int *phys);
int orkan_get_labels(orkan_h h, int *phys);
/* mode 1: orkan_run_circuit first gives the tile's m positions to the m
 * qubits the circuit uses most, when the net number of ops that become
 * in-tile (entering minus leaving) is at least four per swap it costs; the
 * map then stays.  0 (default): never. */
int orkan_set_relabel(orkan_h h, int mode);

/* ------------------------------------------------------------------ packed column-major layout
 * Sec. III-A: the N (N + 1) / 2 lower-triangle elements column by column, h_ij
 * (i >= j) at  j N - j (j - 1) / 2 + (i - j).  The layout the paper compares
 * the tiled one against (Sec. IV), kept for that comparison: one op per pass,
 * each 2^k x 2^k block h_{s,s'} (s >= s') updated by one thread straight from
 * HBM, elements above the diagonal read and written through their stored
 * partners.  The array is the caller's device memory (dev_packed, at least
 * orkan_packed_bytes bytes, in the dtype's element format); calls are
 * asynchronous on cuda_stream (NULL = the legacy default stream).  picture:
 * ORKAN_STATE applies Phi, ORKAN_OBSERVABLE the adjoint Phi*.  Supported: any
 * k = 1 map, k = 2 unitaries (monomial ones without arithmetic); EINVAL for
 * k = 2 Kraus sets with r > 1, k = 3, bad sizes or qubits. */
size_t orkan_packed_bytes(int n, int dtype);
/* Element offset of h_ij in the packed array (host only); *conj = 1 when
 * h_ij is the conjugate of the stored element (i < j).  -1 on bad arguments. */
int64_t orkan_packed_offset(int n, int64_t i, int64_t j, int *conj);
int orkan_packed_apply_unitary(void *dev_packed, int n, int dtype, int picture, int k, const int *qubits,
                               const double *U, void *cuda_stream);
int orkan_packed_apply_kraus(void *dev_packed, int n, int dtype, int picture, int k, const int *qubits, int r,
                             const double *K, void *cuda_stream);
int orkan_packed_depolarize(void *dev_packed, int n, int dtype, int q, double p, void *cuda_stream);
/* Copy h's operator into / out of a packed array of the same n and dtype, on
 * h's stream (pending fused ops are launched first). */
int orkan_packed_from_tiled(orkan_h h, void *dev_packed);
int orkan_packed_to_tiled(orkan_h h, const void *dev_packed);

/* ------------------------------------------------------------------ instrumentation */

/* Counters since allocation: passes launched, ops applied, kernels launched. */
int orkan_stats(orkan_h h, int64_t *passes, int64_t *ops, int64_t *launches);

/* enable != 0: bracket every pass launch with CUDA events on the handle's stream. */
int orkan_set_timing(orkan_h h, int enable);

/* Wait for the stream, then return the summed event time (ms) of the passes
 * recorded since the last call, their count, and reset. */
int orkan_pass_time(orkan_h h, double *ms, int64_t *count);

/* Algorithmic work of the timed passes since the last call, then reset:
 * alu_ops = sum over ops and stored elements of the arithmetic the op's form
 * needs per element (FP32 pipe instructions for C64 and DF64 -- a double-float
 * add is 11, a multiply-add 12 -- FP64 pipe operations for C128; addressing
 * and data movement excluded); bytes = 2 x stored bytes per pass. */
int orkan_pass_work(orkan_h h, double *alu_ops, double *bytes);

/* Measure the current GPU's arithmetic pipes and copy bandwidth (the
 * denominators of ALU and HBM rooflines): out[0] FP32 FMA, out[1] FP64 FMA,
 * out[2] FP32 add, out[3] FP64 add (instructions per second, each from 8
 * independent dependency chains per thread on 8 CTAs per SM), out[4] the read +
 * write bandwidth (GB/s) of a grid-stride copy of 16-byte elements, out[5]
 * paired FP32 FMA (f32x2) in lanes per second (two per instruction; 4 float2
 * chains per thread, the same lane work as out[0]).  out holds 6 values.  scratch:
 * caller-owned device memory, at least 32 MiB (more gives a steadier copy
 * figure; 4 GiB is far beyond the L2).  Blocks for about a second; runs on the
 * legacy default stream.  Not part of any operation's path. */
int orkan_probe_pipes(double *out, void *scratch, size_t scratch_bytes);

/* ------------------------------------------------------------------ allocation-free readout
 * The paper has no counterpart to this entry point; it exists for callers that
 * must not allocate device memory themselves -- e.g. code that runs while a
 * host framework owns all device memory through its own pool and forbids side
 * allocations, serving loops where an allocation could synchronise the device
 * or fail under fragmentation, or plugins that are only handed the device
 * pointer of a tiled operator.
 *
 * tr(P_s H) for count Pauli strings P_s (count * n characters of "IXYZ" back
 * to back).  dev_state is caller-owned device memory holding the array that
 * orkan_device_ptr returns for a handle of this n, dtype and tile_log2, and
 * the strings act on that array's bit positions: character l acts on
 * physical bit position l.  For a handle whose labels are not the identity
 * (orkan_relabel, or the automatic planner), move character q of a logical
 * string to position phys[q] (orkan_get_labels) first.
 *
 * Ordering: the call reads dev_state on cuda_stream (NULL = legacy default
 * stream).  Every write to dev_state must have completed before, or be
 * ordered before cuda_stream by the caller: a handle's stream is a
 * non-blocking stream, so work flushed to it is NOT ordered before the
 * legacy default stream or any other stream.  Either call orkan_sync on the
 * handle first, or record an event on the handle's stream and make
 * cuda_stream wait for it.  The results go to the host array out[count];
 * the call returns after its work on cuda_stream has finished.
 *
 * Scratch: no cudaMalloc / cudaFree or other allocating routine is called.  The
 * partial sums live in one fixed, file-scope device array of
 * ORKAN_NOALLOC_MAX_STRINGS x 608 x 2 + 2 x ORKAN_NOALLOC_MAX_STRINGS doubles
 * (about 609 KB), which every GPU that loads the library holds until the
 * process exits.  count above ORKAN_NOALLOC_MAX_STRINGS is rejected with
 * ORKAN_EINVAL and a message naming the limit.  The array is shared by every
 * call and keeps the last call's contents; each call rewrites every entry it
 * reads, so nothing needs clearing, but calls whose work overlaps on the GPU
 * (other host threads, other streams) race on it and must be serialised by the
 * caller.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) once, with that device current, and keeps it for the
 * life of the process; make that first call before any stream capture.  The
 * kept address does not survive cudaDeviceReset: do not call this entry
 * point on a device after resetting it.
 *
 * Results equal orkan_expect_pauli's bit for bit for the same string (same
 * grid, per-thread order and reduction tree).
 * Errors: EINVAL (null pointers, bad n / dtype / tile_log2, count out of
 * range, bad character), ECUDA. */
#define ORKAN_NOALLOC_MAX_STRINGS 64
int orkan_expect_paulis_noalloc(const void *dev_state, int n, int dtype, int tile_log2, int count,
                                const char *paulis, double *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* ORKAN_H */
