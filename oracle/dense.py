"""Dense complex128 oracle for k-local quantum operations on hermitian operators.

Test infrastructure only: imported by the tests, ``smoke()`` and the CPU
baseline leg of ``bench.py``; never by the CUDA library.

What it computes is the plain definition of the method, written out:

* Eq. (1), Sec. II: ``Phi(H) = sum_alpha K_alpha H K_alpha^dagger`` with every
  ``K_alpha`` built explicitly as the ``N x N`` Kronecker product
  ``I (x) L_alpha (x) I`` of Sec. II-A (k-local factorisation), no blocking,
  no bit tricks, no transfer matrix.
* Sec. I / Sec. II (trace duality): the Heisenberg picture applies the adjoint
  map ``Phi*(O) = sum_alpha K_alpha^dagger O K_alpha``.
* Sec. IV-A: the depolarising channel with Kraus operators
  ``sqrt(1-p) I, sqrt(p/3) X, sqrt(p/3) Y, sqrt(p/3) Z``.
* Dephasing and amplitude damping are not defined in the paper; the textbook
  Kraus sets are used (``sqrt(1-p) I, sqrt(p) Z`` and
  ``diag(1, sqrt(1-g)), sqrt(g)|0><1|``).
* Measurement in the Z basis is a pair of projectors ``Pi_0, Pi_1`` (a trace
  non-increasing map, Sec. II) followed by Born renormalisation.

Conventions (shared with the library only as a documented convention, never
as code): qubit ``a`` is bit ``a`` of a basis index (qubit 0 is the least
significant bit, as in the swap rule of Sec. II-B and Subroutine 1); a
``2^k x 2^k`` operator ``L`` given on the qubit list ``qubits`` maps bit ``l``
of its own index to qubit ``qubits[l]``.

Dense embeddings are used for ``n <= DENSE_MAX_N``; above that the same
Kronecker products are formed with ``scipy.sparse`` (CSR), which computes the
identical matrix without storing its zeros.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

DENSE_MAX_N = 8

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULI = {"I": I2, "X": X, "Y": Y, "Z": Z}


# --------------------------------------------------------------------------
# Embedding of a k-local operator (Sec. II-A: K = I (x) L)
# --------------------------------------------------------------------------
def _qubit_permutation_matrix(n: int, qubits, sparse: bool):
    """Basis permutation P with P|x> = |pi(x)>, where pi moves bit l of x to
    position ``qubits[l]`` for l < k and the remaining bits, in increasing
    order, to the remaining positions in increasing order."""
    k = len(qubits)
    rest = [p for p in range(n) if p not in qubits]
    dest = list(qubits) + rest  # bit l of the standard order goes to dest[l]
    N = 1 << n
    src = np.arange(N)
    tgt = np.zeros(N, dtype=np.int64)
    for l in range(n):
        tgt |= ((src >> l) & 1) << dest[l]
    if sparse:
        return sp.csr_matrix((np.ones(N, dtype=np.complex128), (tgt, src)), shape=(N, N))
    P = np.zeros((N, N), dtype=np.complex128)
    P[tgt, src] = 1.0
    assert k <= n
    return P


def embed(L: np.ndarray, qubits, n: int, sparse: bool | None = None):
    """Return ``K = I (x) L (x) I`` on ``n`` qubits for ``L`` acting on
    ``qubits`` (bit l of L's index <-> qubit ``qubits[l]``).

    A single qubit ``a`` gives ``kron(I_{2^(n-1-a)}, L, I_{2^a})``.  For any
    other qubit list the operator is first embedded on qubits ``0..k-1`` as
    ``kron(I_{2^(n-k)}, L)`` and then conjugated by the explicit basis
    permutation that moves qubit ``l`` to ``qubits[l]``.
    """
    qubits = [int(q) for q in qubits]
    k = len(qubits)
    L = np.asarray(L, dtype=np.complex128)
    assert L.shape == (1 << k, 1 << k)
    assert len(set(qubits)) == k and all(0 <= q < n for q in qubits)
    if sparse is None:
        sparse = n > DENSE_MAX_N
    kron = sp.kron if sparse else np.kron
    eye = (lambda d: sp.identity(d, dtype=np.complex128, format="csr")) if sparse else (
        lambda d: np.eye(d, dtype=np.complex128))
    if k == 1:
        a = qubits[0]
        K = kron(kron(eye(1 << (n - 1 - a)), L), eye(1 << a))
        return sp.csr_matrix(K) if sparse else K
    K0 = kron(eye(1 << (n - k)), L)
    P = _qubit_permutation_matrix(n, qubits, sparse)
    K = P @ K0 @ P.conj().T
    return sp.csr_matrix(K) if sparse else K


def _left(K, H):
    """K @ H for dense or sparse K, dense result."""
    R = K @ H
    return np.asarray(R.todense()) if sp.issparse(R) else np.asarray(R)


def _conjugate(K, H):
    """K H K^dagger with the products evaluated as written."""
    KH = _left(K, H)
    # (K H) K^dagger = (K (K H)^dagger)^dagger
    return _left(K, KH.conj().T).conj().T


def _conjugate_adjoint(K, H):
    """K^dagger H K."""
    Kd = K.conj().T
    return _conjugate(sp.csr_matrix(Kd) if sp.issparse(K) else Kd, H)


# --------------------------------------------------------------------------
# Eq. (1): the Kraus map and its adjoint
# --------------------------------------------------------------------------
def apply_kraus(H: np.ndarray, kraus, qubits, picture: str = "schrodinger") -> np.ndarray:
    """Eq. (1): ``H <- sum_alpha K_alpha H K_alpha^dagger`` (Schroedinger) or
    the trace-dual ``H <- sum_alpha K_alpha^dagger H K_alpha`` (Heisenberg)."""
    n = int(np.log2(H.shape[0]))
    out = np.zeros_like(H, dtype=np.complex128)
    for L in kraus:
        K = embed(L, qubits, n)
        if picture == "schrodinger":
            out += _conjugate(K, H)
        elif picture == "heisenberg":
            out += _conjugate_adjoint(K, H)
        else:
            raise ValueError(picture)
    return out


def apply_unitary(H, U, qubits, picture="schrodinger"):
    """A unitary gate is the Kraus map with the single operator U."""
    return apply_kraus(H, [U], qubits, picture)


# --------------------------------------------------------------------------
# Named channels (Kraus sets)
# --------------------------------------------------------------------------
def depolarizing_kraus(p: float):
    """Sec. IV-A: sqrt(1-p) I, sqrt(p/3) X, sqrt(p/3) Y, sqrt(p/3) Z."""
    return [np.sqrt(1 - p) * I2, np.sqrt(p / 3) * X, np.sqrt(p / 3) * Y, np.sqrt(p / 3) * Z]


def dephasing_kraus(p: float):
    """Textbook phase flip: sqrt(1-p) I, sqrt(p) Z (not defined in the paper)."""
    return [np.sqrt(1 - p) * I2, np.sqrt(p) * Z]


def amplitude_damping_kraus(gamma: float):
    """Textbook amplitude damping (not defined in the paper):
    K0 = diag(1, sqrt(1-g)), K1 = sqrt(g) |0><1|."""
    K0 = np.array([[1, 0], [0, np.sqrt(1 - gamma)]], dtype=np.complex128)
    K1 = np.array([[0, np.sqrt(gamma)], [0, 0]], dtype=np.complex128)
    return [K0, K1]


def depolarize(H, q, p, picture="schrodinger"):
    return apply_kraus(H, depolarizing_kraus(p), [q], picture)


def dephase(H, q, p, picture="schrodinger"):
    return apply_kraus(H, dephasing_kraus(p), [q], picture)


def amplitude_damp(H, q, gamma, picture="schrodinger"):
    return apply_kraus(H, amplitude_damping_kraus(gamma), [q], picture)


# --------------------------------------------------------------------------
# Measurement (projectors, a CP-TNI map of Sec. II) and Born renormalisation
# --------------------------------------------------------------------------
def projector(b: int) -> np.ndarray:
    P = np.zeros((2, 2), dtype=np.complex128)
    P[b, b] = 1.0
    return P


def born_probabilities(H, q):
    """p_b = Re tr(Pi_b H) for b = 0, 1, with Pi_b = I (x) |b><b| (x) I."""
    n = int(np.log2(H.shape[0]))
    ps = []
    for b in (0, 1):
        Pi = embed(projector(b), [q], n)
        ps.append(float(np.real(np.trace(_left(Pi, H)))))
    return ps[0], ps[1]


def measure(H, q, u):
    """Z-basis measurement of qubit q with the uniform draw u in [0, 1).

    outcome 0 iff u < p0 / (p0 + p1); then H <- Pi_b H Pi_b / p_b.
    Returns (H', outcome, p_b / (p0 + p1))."""
    p0, p1 = born_probabilities(H, q)
    tot = p0 + p1
    b = 0 if u * tot < p0 else 1
    pb = (p0, p1)[b]
    if not pb > 1e-300:
        raise ZeroDivisionError("zero-probability outcome")
    Hp = apply_kraus(H, [projector(b)], [q]) / pb
    return Hp, b, pb / tot


def project(H, q, b):
    """Pi_b H Pi_b without renormalisation: the single-Kraus trace
    non-increasing map of Sec. II with K = Pi_b, which is self-adjoint, so
    both pictures apply the same map."""
    return apply_kraus(H, [projector(b)], [q])


# --------------------------------------------------------------------------
# Readouts
# --------------------------------------------------------------------------
def pauli_matrix(pauli: str) -> np.ndarray:
    """Dense Pauli string; character l acts on qubit l (bit l of the index)."""
    P = np.ones((1, 1), dtype=np.complex128)
    for ch in reversed(pauli):  # qubit n-1 is the leftmost Kronecker factor
        P = np.kron(P, PAULI[ch])
    return P


def pauli_sum(paulis, coeffs) -> np.ndarray:
    """O = sum_t coeffs[t] P_t, the observable evolved in the Heisenberg
    picture (Sec. I: predictions tr(rho O) are the same in both pictures)."""
    n = len(paulis[0])
    O = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for s, c in zip(paulis, coeffs):
        O += c * pauli_matrix(s)
    return O


def expect_pauli(H, pauli: str) -> complex:
    """tr(P H)."""
    return complex(np.trace(pauli_matrix(pauli) @ H))


def expect(rho, O) -> complex:
    """tr(rho O), the prediction of Sec. I."""
    return complex(np.trace(rho @ O))


def trace(H) -> complex:
    return complex(np.trace(H))


# --------------------------------------------------------------------------
# Circuits (a list of op dicts produced by workloads.synth)
# --------------------------------------------------------------------------
def apply_op(H, op, picture="schrodinger"):
    """Apply one op dict; returns (H', record) where record holds measurement
    outcomes for ops of kind 'measure'."""
    kind = op["kind"]
    if kind == "unitary":
        return apply_unitary(H, op["matrix"], op["qubits"], picture), None
    if kind == "kraus":
        return apply_kraus(H, op["mats"], op["qubits"], picture), None
    if kind == "depolarize":
        return depolarize(H, op["qubits"][0], op["p"], picture), None
    if kind == "dephase":
        return dephase(H, op["qubits"][0], op["p"], picture), None
    if kind == "ampdamp":
        return amplitude_damp(H, op["qubits"][0], op["gamma"], picture), None
    if kind == "measure":
        if picture == "schrodinger":
            Hp, b, pb = measure(H, op["qubits"][0], op["u"])
            return Hp, (b, pb)
        b = 0 if op["u"] < 0.5 else 1
        return project(H, op["qubits"][0], b), (b, None)
    if kind == "project":
        return project(H, op["qubits"][0], op["outcome"]), None
    raise ValueError(kind)


def run_circuit(H, ops, picture="schrodinger"):
    records = []
    for op in ops:
        H, rec = apply_op(H, op, picture)
        if rec is not None:
            records.append(rec)
    return H, records


# --------------------------------------------------------------------------
# Error measures
# --------------------------------------------------------------------------
def max_abs_diff(A, B) -> float:
    return float(np.max(np.abs(np.asarray(A) - np.asarray(B))))


def frobenius_diff(A, B) -> float:
    return float(np.linalg.norm(np.asarray(A) - np.asarray(B)))


def trace_distance(A, B) -> float:
    """0.5 ||A - B||_1 for hermitian A, B (eigenvalues of the difference)."""
    D = np.asarray(A) - np.asarray(B)
    D = 0.5 * (D + D.conj().T)
    return float(0.5 * np.sum(np.abs(np.linalg.eigvalsh(D))))


# --------------------------------------------------------------------------
# Eq. (1) on a factored operator (for sampled checks at large n)
# --------------------------------------------------------------------------
def apply_kraus_to_factors(vectors, kraus, qubits, n):
    """For H = sum_v v v^dagger, Eq. (1) gives Phi(H) = sum_alpha sum_v
    (K_alpha v)(K_alpha v)^dagger; return the list of all K_alpha v.  Each
    K_alpha is the same explicit (sparse above DENSE_MAX_N) Kronecker
    embedding used by :func:`apply_kraus`."""
    out = []
    for L in kraus:
        K = embed(L, qubits, n)
        for v in vectors:
            out.append(np.asarray(K @ v).reshape(-1))
    return out


def factored_elements(vectors, rows, cols):
    """H[rows[t], cols[t]] of H = sum_v v v^dagger."""
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    out = np.zeros(rows.shape, dtype=np.complex128)
    for v in vectors:
        out += v[rows] * np.conj(v[cols])
    return out
