"""Seeded generators for states, observables and circuits.

Every generator takes an explicit seed (NumPy PCG64).  The base seed of
workload ``c`` is ``20260415 + c``.  The recipes follow the workloads the
paper benchmarks (random hermitian operators, single-qubit channels swept over
all targets, Sec. IV-A) widened to the circuit mixes used for parity and
throughput:

* ``config0``: n=8, Ginibre state ``W W^dagger / tr W W^dagger``, 200 ops
  (40 % Haar 1-qubit U, 30 % Haar 2-qubit U on an ordered distinct pair,
  10 % depolarising p~U[0,0.05], 10 % amplitude damping g~U[0,0.1],
  10 % Z measurement with a uniform draw u), then 8 Pauli strings.
* ``sweep``: every op class on every target (the per-op sweep).
* ``brickwork``: layered noisy brickwork circuit.
* ``serving_stream``: Poisson arrivals of mixed-size requests.

An op is a dict ``{"kind": ..., "qubits": [...], ...}``; kinds are
``unitary`` (``matrix``), ``kraus`` (``mats``), ``depolarize`` (``p``),
``dephase`` (``p``), ``ampdamp`` (``gamma``), ``measure`` (``u``) and
``project`` (``outcome``).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20260415


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# random matrices
# --------------------------------------------------------------------------
def haar_unitary(rng: np.random.Generator, d: int) -> np.ndarray:
    """Haar-random unitary: QR of a complex Ginibre matrix with the phases of
    R's diagonal moved into Q (Mezzadri, Notices AMS 54, 2007)."""
    Zm = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Zm)
    ph = np.diag(R) / np.abs(np.diag(R))
    return (Q * ph[None, :]).astype(np.complex128)


def ginibre_state(rng: np.random.Generator, N: int) -> np.ndarray:
    """rho = W W^dagger / tr(W W^dagger), W with i.i.d. complex normal entries."""
    W = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    rho = W @ W.conj().T
    rho = 0.5 * (rho + rho.conj().T)
    return (rho / np.trace(rho).real).astype(np.complex128)


def random_hermitian(rng: np.random.Generator, N: int) -> np.ndarray:
    """Hermitian, neither PSD nor normalised (the benchmark operator of Sec. IV-A)."""
    A = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    return (0.5 * (A + A.conj().T)).astype(np.complex128)


def haar_state_vector(rng: np.random.Generator, N: int) -> np.ndarray:
    v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    return (v / np.linalg.norm(v)).astype(np.complex128)


def random_product_vector(rng: np.random.Generator, n: int) -> np.ndarray:
    """Tensor product of n Haar-random single-qubit pure states (qubit 0 is the
    least significant index bit)."""
    v = np.ones(1, dtype=np.complex128)
    for _ in range(n):
        q = haar_state_vector(rng, 2)
        v = np.kron(q, v)
    return v


def random_pauli_strings(rng: np.random.Generator, n: int, count: int, allow_identity=True):
    out = []
    while len(out) < count:
        s = "".join("IXYZ"[int(c)] for c in rng.integers(0, 4, size=n))
        if not allow_identity and set(s) == {"I"}:
            continue
        out.append(s)
    return out


def random_pauli_sum(rng: np.random.Generator, n: int, nterms: int = 16):
    """nterms Pauli strings with real coefficients ~ N(0, 1)."""
    strings = random_pauli_strings(rng, n, nterms)
    coeffs = rng.standard_normal(nterms)
    return strings, coeffs


# --------------------------------------------------------------------------
# op constructors
# --------------------------------------------------------------------------
def op_unitary(U, qubits):
    return {"kind": "unitary", "qubits": [int(q) for q in qubits], "matrix": np.asarray(U, np.complex128)}


def op_kraus(mats, qubits):
    return {"kind": "kraus", "qubits": [int(q) for q in qubits], "mats": [np.asarray(K, np.complex128) for K in mats]}


def op_depolarize(q, p):
    return {"kind": "depolarize", "qubits": [int(q)], "p": float(p)}


def op_dephase(q, p):
    return {"kind": "dephase", "qubits": [int(q)], "p": float(p)}


def op_ampdamp(q, gamma):
    return {"kind": "ampdamp", "qubits": [int(q)], "gamma": float(gamma)}


def op_measure(q, u):
    return {"kind": "measure", "qubits": [int(q)], "u": float(u)}


def op_project(q, outcome):
    return {"kind": "project", "qubits": [int(q)], "outcome": int(outcome)}


# --------------------------------------------------------------------------
# circuits
# --------------------------------------------------------------------------
def random_mixed_circuit(rng: np.random.Generator, n: int, depth: int, with_measure=True):
    """The op mix of the n=8 parity workload: 40/30/10/10/10 %."""
    ops = []
    probs = np.array([0.4, 0.3, 0.1, 0.1, 0.1])
    if not with_measure:
        probs = np.array([0.4, 0.3, 0.15, 0.15, 0.0])
    for _ in range(depth):
        c = int(rng.choice(5, p=probs))
        if c == 0:
            ops.append(op_unitary(haar_unitary(rng, 2), [int(rng.integers(n))]))
        elif c == 1 and n >= 2:
            a, b = rng.choice(n, size=2, replace=False)
            ops.append(op_unitary(haar_unitary(rng, 4), [int(a), int(b)]))
        elif c == 1:
            ops.append(op_unitary(haar_unitary(rng, 2), [0]))
        elif c == 2:
            ops.append(op_depolarize(int(rng.integers(n)), rng.uniform(0.0, 0.05)))
        elif c == 3:
            ops.append(op_ampdamp(int(rng.integers(n)), rng.uniform(0.0, 0.1)))
        else:
            ops.append(op_measure(int(rng.integers(n)), rng.uniform(0.0, 1.0)))
    return ops


def config0(seed: int = BASE_SEED + 0, n: int = 8, depth: int = 200):
    """n=8 parity workload: Ginibre state, 200 mixed ops, 8 Pauli strings."""
    rng = rng_for(seed)
    rho = ginibre_state(rng, 1 << n)
    ops = random_mixed_circuit(rng, n, depth)
    paulis = random_pauli_strings(rng, n, 8)
    return {"n": n, "rho": rho, "ops": ops, "paulis": paulis}


def sweep(n: int, seed: int = BASE_SEED + 1, p_depol=0.1, gamma=0.05):
    """Per-op sweep: for every target q, a Haar 1-qubit U, depolarising
    (4 Kraus, p), amplitude damping (2 Kraus, gamma), and Haar 2-qubit U on the
    adjacent pair (q, q+1 mod n) and the far pair (q, n-1-q) when distinct."""
    rng = rng_for(seed)
    ops = []
    for q in range(n):
        ops.append(op_unitary(haar_unitary(rng, 2), [q]))
        ops.append(op_depolarize(q, p_depol))
        ops.append(op_ampdamp(q, gamma))
        if n >= 2:
            ops.append(op_unitary(haar_unitary(rng, 4), [q, (q + 1) % n]))
            if n - 1 - q != q:
                ops.append(op_unitary(haar_unitary(rng, 4), [q, n - 1 - q]))
    return ops


def brickwork(n: int, depth: int, seed: int = BASE_SEED + 2, p_depol=1e-3):
    """Layered noisy brickwork: per layer a Haar 1-qubit U on every qubit, Haar
    2-qubit U on (0,1),(2,3),... (even layers) or (1,2),(3,4),... (odd layers),
    then depolarising p on every qubit."""
    rng = rng_for(seed)
    ops = []
    for layer in range(depth):
        for q in range(n):
            ops.append(op_unitary(haar_unitary(rng, 2), [q]))
        start = layer % 2
        for q in range(start, n - 1, 2):
            ops.append(op_unitary(haar_unitary(rng, 4), [q, q + 1]))
        for q in range(n):
            ops.append(op_depolarize(q, p_depol))
    return ops


def serving_stream(count: int = 5000, seed: int = BASE_SEED + 4, rate: float = 1000.0,
                   n_range=(4, 14), depth_range=(10, 200)):
    """Poisson request stream: arrival times (s), n ~ U{4..14}, depth ~
    U{10..200} from the mixed op mix, picture and dtype 50/50.  Schroedinger
    requests start from a random product state and read 8 Pauli strings;
    Heisenberg requests evolve a 16-term Pauli sum and read tr(O rho0) for a
    random product state rho0."""
    rng = rng_for(seed)
    t = 0.0
    reqs = []
    for rid in range(count):
        t += rng.exponential(1.0 / rate)
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        depth = int(rng.integers(depth_range[0], depth_range[1] + 1))
        picture = "schrodinger" if rng.uniform() < 0.5 else "heisenberg"
        dtype = "c128" if rng.uniform() < 0.5 else "c64"
        ops = random_mixed_circuit(rng, n, depth, with_measure=(picture == "schrodinger"))
        req = {"id": rid, "t": t, "n": n, "depth": depth, "picture": picture, "dtype": dtype, "ops": ops}
        if picture == "schrodinger":
            req["psi0"] = random_product_vector(rng, n)
            req["paulis"] = random_pauli_strings(rng, n, 8)
        else:
            req["paulis"], req["coeffs"] = random_pauli_sum(rng, n, 16)
            req["psi0"] = random_product_vector(rng, n)
        reqs.append(req)
    return reqs
