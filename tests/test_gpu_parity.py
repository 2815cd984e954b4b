"""GPU parity: the CUDA path, called through the C ABI, against the oracle.

Every comparison is element by element on the same seeded inputs.
Tolerances on max |delta H_ij|:
  c128 (native FP64) and df64 (double-float, ~48 significand bits):
      1e-12 * max(1, max |H_ij|)  (the stated bound for unit-trace states),
      and at large n also 1e-10 * max |H_ij| (relative to the operator's scale)
  c64 (FP32 storage and arithmetic): 1e-5 * max |H_ij|
Measurement outcomes must agree exactly (both sides decide in FP64; the
workloads are checked to keep every draw u at least 1e-6 away from the
threshold p0 / (p0 + p1)).
"""
import itertools

import numpy as np
import pytest

from oracle import dense as D
from oracle import tiled as T
from workloads import synth as S

pytestmark = pytest.mark.gpu

ok = pytest.importorskip("paper_2604_15765_gb300.orkan")
from paper_2604_15765_gb300 import circuit  # noqa: E402

TOL = {"c128": 1e-12, "df64": 1e-12, "c64": 1e-5}
REL_BIG = {"c128": 1e-10, "df64": 1e-10, "c64": 1e-4}
DT = {"c128": 0, "c64": 1, "df64": 2}


def _tol(name, ref):
    scale = float(np.max(np.abs(ref)))
    return TOL[name] * (scale if name == "c64" else max(1.0, scale))


def _handle(n, dtype, m=5, fusion=8, compose=True):
    h = ok.orkan_alloc(n, DT[dtype], m)
    ok.orkan_set_fusion(h, fusion, compose)
    return h


def _assert_close(got, ref, dtype, what="", rel=None):
    err = np.max(np.abs(got - ref))
    assert err <= _tol(dtype, ref), f"{what}: max|delta| = {err:.3e} > {_tol(dtype, ref):.1e}"
    if rel is not None:
        scale = float(np.max(np.abs(ref)))
        assert err <= rel * scale, f"{what}: max|delta| = {err:.3e} > {rel:.0e} * {scale:.3e}"
    return err


# ------------------------------------------------------------------ single ops, every target
def _single_ops(n, rng):
    """Every op class on every target / pair for an n-qubit operator."""
    ops = []
    for q in range(n):
        ops.append(S.op_unitary(S.haar_unitary(rng, 2), [q]))
        ops.append(S.op_depolarize(q, 0.1))
        ops.append(S.op_ampdamp(q, 0.05))
        ops.append(S.op_dephase(q, 0.2))
        ks = [rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2)) for _ in range(3)]
        ops.append(S.op_kraus([0.4 * k for k in ks], [q]))
        ops.append(S.op_project(q, q & 1))
    if n >= 2:
        pairs = set()
        for q in range(n):
            pairs.add((q, (q + 1) % n))
            pairs.add(((q + 1) % n, q))
            if n - 1 - q != q:
                pairs.add((q, n - 1 - q))
        for a, b in sorted(pairs):
            ops.append(S.op_unitary(S.haar_unitary(rng, 4), [a, b]))
        for a, b in sorted(pairs)[:: max(1, len(pairs) // 6)]:
            ks = [rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)) for _ in range(2)]
            ops.append(S.op_kraus([0.3 * k for k in ks], [a, b]))
    return ops


CASES = [(n, 5) for n in range(1, 9)] + [(6, 3), (7, 3), (8, 3), (7, 4), (9, 3), (9, 4)]


@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
@pytest.mark.parametrize("picture", ["schrodinger", "heisenberg"])
@pytest.mark.parametrize("n,m", CASES)
def test_single_op_every_target(n, m, dtype, picture):
    rng = S.rng_for(1000 + 31 * n + m)
    N = 1 << n
    if picture == "schrodinger":
        H0 = S.ginibre_state(rng, N)
    else:
        strings, coeffs = S.random_pauli_sum(rng, n, 16)
        H0 = D.pauli_sum(strings, coeffs)
    tiled0 = T.to_tiled(H0, m)
    h = _handle(n, dtype, m, fusion=1, compose=False)
    try:
        for op in _single_ops(n, rng):
            if dtype == "c128":
                ok.orkan_load_tiled(h, tiled0, 0 if picture == "schrodinger" else 1)
            else:
                if picture == "schrodinger":
                    ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, H0)
                else:
                    ok.orkan_init_observable(h, strings, coeffs)
            circuit.apply_op(h, op, picture)
            got = ok.orkan_to_dense(h)
            ref, _ = D.apply_op(H0, op, picture)
            _assert_close(got, ref, dtype, f"{op['kind']} on {op['qubits']}")
    finally:
        ok.orkan_free(h)


# ------------------------------------------------------------------ the n = 8 circuit workload
@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
@pytest.mark.parametrize("fusion", [(1, False), (8, True), (16, True)])
def test_config0_circuit_n8(dtype, fusion):
    w = S.config0()
    n, rho0, ops = w["n"], w["rho"], w["ops"]
    ref, recs = D.run_circuit(rho0, ops)
    # every measurement draw is well away from its threshold
    rho = rho0
    for op in ops:
        if op["kind"] == "measure":
            p0, p1 = D.born_probabilities(rho, op["qubits"][0])
            assert abs(op["u"] - p0 / (p0 + p1)) > 1e-6
        rho, _ = D.apply_op(rho, op)
    h = _handle(n, dtype, 5, *fusion)
    try:
        ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, rho0)
        got_recs = circuit.run_circuit(h, ops)
        assert [b for b, _ in got_recs] == [b for b, _ in recs]
        for (_, pg), (_, pr) in zip(got_recs, recs):
            assert abs(pg - pr) <= TOL[dtype] * 10
        got = ok.orkan_to_dense(h)
        err = _assert_close(got, ref, dtype, "config0 final state")
        for s in w["paulis"]:
            e_ref = D.expect_pauli(ref, s).real
            assert abs(ok.orkan_expect_pauli(h, s) - e_ref) <= TOL[dtype] * 10, s
        tr = ok.orkan_trace(h)
        assert abs(tr - 1.0) <= TOL[dtype] * 10
        print(f"config0 {dtype} fusion={fusion}: max|delta| = {err:.3e}")
    finally:
        ok.orkan_free(h)


# ------------------------------------------------------------------ fused passes (h = 0, 1, 2 with low ops)
@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
@pytest.mark.parametrize("n,m", [(8, 3), (9, 4), (7, 5), (10, 3)])
def test_fused_random_circuit(n, m, dtype):
    rng = S.rng_for(2000 + n + 10 * m)
    rho0 = S.ginibre_state(rng, 1 << n)
    ops = S.random_mixed_circuit(rng, n, 60, with_measure=False)
    for q in range(min(n, 3)):   # ops on low qubits mixed with high pairs
        ops.append(S.op_unitary(S.haar_unitary(rng, 2), [q]))
        ops.append(S.op_unitary(S.haar_unitary(rng, 4), [n - 1, n - 2]))
    ref, _ = D.run_circuit(rho0, ops)
    for fusion in ((16, True), (16, False), (1, False)):
        h = _handle(n, dtype, m, *fusion)
        try:
            ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, rho0)
            circuit.run_circuit(h, ops)
            _assert_close(ok.orkan_to_dense(h), ref, dtype, f"fusion {fusion}")
            st = ok.orkan_stats(h)
            if fusion[0] == 1:
                assert st["passes"] == len(ops)
            else:
                assert st["passes"] < len(ops)
        finally:
            ok.orkan_free(h)


# ------------------------------------------------------------------ chunked passes with many diagonal groups
@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
@pytest.mark.parametrize("n", [9, 10, 11])
def test_chunked_high_pairs(n, dtype):
    """Two high qubits in one pass at m = 5 split tiles into row chunks; the
    diagonal tile groups then run in the full-height diagonal kernel.  Mixed
    ops (low ones fused in, high pairs in both orders, 2-qubit Kraus maps)."""
    rng = S.rng_for(2500 + n)
    rho0 = S.ginibre_state(rng, 1 << n)
    ops = []
    for a, b in [(n - 1, n - 2), (5, n - 1), (6, 5), (n - 3, n - 1), (8, 5)]:
        ops.append(S.op_unitary(S.haar_unitary(rng, 2), [a % 3]))
        ops.append(S.op_unitary(S.haar_unitary(rng, 4), [a, b]))
        ops.append(S.op_unitary(S.haar_unitary(rng, 4), [b % 3, a]))
        ops.append(S.op_depolarize(b, 0.07))
        ks = [rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)) for _ in range(2)]
        ops.append(S.op_kraus([0.3 * k for k in ks], [b, a]))
    ref, _ = D.run_circuit(rho0, ops)
    for fusion in ((8, True), (1, False)):
        h = _handle(n, dtype, 5, *fusion)
        try:
            ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, rho0)
            circuit.run_circuit(h, ops)
            _assert_close(ok.orkan_to_dense(h), ref, dtype, f"fusion {fusion}", rel=REL_BIG[dtype])
        finally:
            ok.orkan_free(h)


# ------------------------------------------------------------------ init kinds and layout
@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
@pytest.mark.parametrize("n,m", [(1, 5), (3, 3), (5, 5), (7, 3), (9, 5)])
def test_init_kinds_and_layout(n, m, dtype):
    rng = S.rng_for(3000 + n * 7 + m)
    N = 1 << n
    h = _handle(n, dtype, m)
    try:
        ok.orkan_init_state(h, ok.ORKAN_INIT_ZERO)
        ref = np.zeros((N, N), dtype=np.complex128)
        ref[0, 0] = 1
        assert np.array_equal(ok.orkan_to_dense(h), ref)
        ok.orkan_init_state(h, ok.ORKAN_INIT_MAXMIXED)
        _assert_close(ok.orkan_to_dense(h), np.eye(N) / N, dtype, "maxmixed")
        psi = S.haar_state_vector(rng, N)
        ok.orkan_init_state(h, ok.ORKAN_INIT_PURE, psi)
        _assert_close(ok.orkan_to_dense(h), np.outer(psi, psi.conj()), dtype, "pure")
        H = S.random_hermitian(rng, N)
        ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, H)
        _assert_close(ok.orkan_to_dense(h), H, dtype, "dense")
        if dtype == "c128":
            buf = np.empty(T.stored_elements(n, m), dtype=np.complex128)
            ok.orkan_store_tiled(h, buf)
            assert np.array_equal(buf, T.to_tiled(np.tril(H) + np.tril(H, -1).conj().T, m))
        strings, coeffs = S.random_pauli_sum(rng, n, 12)
        strings += ["Y" * n, "X" * n, "I" * n]
        coeffs = np.concatenate([coeffs, [0.5, -0.25, 2.0]])
        ok.orkan_init_observable(h, strings, coeffs)
        _assert_close(ok.orkan_to_dense(h), D.pauli_sum(strings, coeffs), dtype, "pauli sum")
        assert ok.orkan_get_info(h)[3] == ok.ORKAN_OBSERVABLE
    finally:
        ok.orkan_free(h)


# ------------------------------------------------------------------ readouts
@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
@pytest.mark.parametrize("n,m", [(1, 5), (3, 3), (6, 5), (8, 3), (10, 5)])
def test_readouts(n, m, dtype):
    rng = S.rng_for(4000 + n + m)
    N = 1 << n
    rho = S.ginibre_state(rng, N)
    strings, coeffs = S.random_pauli_sum(rng, n, 16)
    O = D.pauli_sum(strings, coeffs)
    hr, ho = _handle(n, dtype, m), _handle(n, dtype, m)
    try:
        ok.orkan_init_state(hr, ok.ORKAN_INIT_DENSE, rho)
        ok.orkan_init_observable(ho, strings, coeffs)
        tr = ok.orkan_trace(hr)
        assert abs(tr - np.trace(rho)) <= TOL[dtype] * 10
        for s in S.random_pauli_strings(rng, n, 12) + ["Y" * n, "Z" * n, "I" * n]:
            assert abs(ok.orkan_expect_pauli(hr, s) - D.expect_pauli(rho, s).real) <= TOL[dtype] * 10, s
        e = ok.orkan_expect(hr, ho)
        assert abs(e - D.expect(rho, O).real) <= TOL[dtype] * 10 * max(1, np.abs(O).max())
        rows = rng.integers(0, N, 200)
        cols = rng.integers(0, N, 200)
        _assert_close(ok.orkan_get_elements(hr, rows, cols), rho[rows, cols], dtype, "gather")
    finally:
        ok.orkan_free(hr)
        ok.orkan_free(ho)


def test_duality_on_gpu():
    """tr(O Phi(rho)) = tr(Phi*(O) rho) with both sides evolved on the GPU."""
    n = 10
    rng = S.rng_for(4500)
    ops = S.random_mixed_circuit(rng, n, 40, with_measure=False)
    rho = S.ginibre_state(rng, 1 << n)
    strings, coeffs = S.random_pauli_sum(rng, n, 16)
    for dtype in ("c128", "df64"):
        hr, ho, h0 = _handle(n, dtype), _handle(n, dtype), _handle(n, dtype)
        try:
            ok.orkan_init_state(hr, ok.ORKAN_INIT_DENSE, rho)
            ok.orkan_init_state(h0, ok.ORKAN_INIT_DENSE, rho)
            ok.orkan_init_observable(ho, strings, coeffs)
            circuit.run_circuit(hr, ops, "schrodinger")
            circuit.run_circuit(ho, list(reversed(ops)), "heisenberg")
            lhs = ok.orkan_expect(hr, _obs(n, dtype, strings, coeffs))
            rhs = ok.orkan_expect(h0, ho)
            assert abs(lhs - rhs) < 1e-11
        finally:
            for x in (hr, ho, h0):
                ok.orkan_free(x)


_OBS_CACHE = {}


def _obs(n, dtype, strings, coeffs):
    key = (n, dtype)
    if key not in _OBS_CACHE:
        h = _handle(n, dtype)
        ok.orkan_init_observable(h, strings, coeffs)
        _OBS_CACHE[key] = h
    return _OBS_CACHE[key]


# ------------------------------------------------------------------ errors and edge cases
def test_errors_and_edge_cases():
    h = _handle(4, "c128")
    try:
        ok.orkan_init_state(h, ok.ORKAN_INIT_ZERO)
        with pytest.raises(ok.OrkanError) as e:
            ok.orkan_apply_unitary(h, [4], np.eye(2))
        assert e.value.status == ok.ORKAN_EINVAL
        with pytest.raises(ok.OrkanError):
            ok.orkan_apply_unitary(h, [1, 1], np.eye(4))
        with pytest.raises(ok.OrkanError):
            ok.orkan_apply_kraus(h, [0], np.zeros((0, 2, 2)))
        with pytest.raises(ok.OrkanError):
            ok.orkan_expect_pauli(h, "XYZQ")
        with pytest.raises(ok.OrkanError):
            ok.orkan_measure(h, 0, 1.0)
        # empty circuit: the state is unchanged
        ok.orkan_flush(h)
        ref = np.zeros((16, 16), dtype=np.complex128)
        ref[0, 0] = 1
        assert np.array_equal(ok.orkan_to_dense(h), ref)
        # |0><0| measured: outcome 0 with probability 1; project to 1 -> zero operator
        assert ok.orkan_measure(h, 2, 0.999) == (0, 1.0)
        ok.orkan_project(h, 0, 1)
        with pytest.raises(ok.OrkanError) as e:
            ok.orkan_measure(h, 0, 0.3)
        assert e.value.status == ok.ORKAN_EZEROPROB
        ok.orkan_init_observable(h, ["ZIII"], [1.0])
        with pytest.raises(ok.OrkanError) as e:
            ok.orkan_measure(h, 0, 0.3)
        assert e.value.status == ok.ORKAN_EPICTURE
    finally:
        ok.orkan_free(h)


def test_pauli_x_is_exact_on_gpu():
    """Sec. II-B: X conjugation only permutes entries; in native FP64 the
    result is the oracle's swap bit for bit (products with 0 and 1 are exact)."""
    n, m = 7, 3
    rng = S.rng_for(4600)
    H = S.random_hermitian(rng, 1 << n)
    h = _handle(n, "c128", m, fusion=1, compose=False)
    try:
        for a in range(n):
            ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, H)
            ok.orkan_apply_unitary(h, [a], D.X)
            perm = np.arange(1 << n) ^ (1 << a)
            ref = H[np.ix_(perm, perm)]
            assert np.max(np.abs(ok.orkan_to_dense(h) - ref)) <= 1e-15 * np.abs(H).max()
    finally:
        ok.orkan_free(h)


# ------------------------------------------------------------------ full sizes, sampled
def _sample_idx(rng, N, count):
    rows = rng.integers(0, N, count)
    cols = rng.integers(0, N, count)
    diag = rng.integers(0, N, count // 8)
    return np.concatenate([rows, diag]), np.concatenate([cols, diag])


@pytest.mark.parametrize("n,dtype", [(14, "c128"), (14, "df64"), (14, "c64"), (16, "df64"), (16, "c128"),
                                     (17, "c64")])
def test_full_size_sampled(n, dtype):
    """The per-op sweep workload at full size in the bench's launch
    configuration (m = 5, fusion 8 with composition).  The input is a Haar
    pure state so that the oracle can compute sampled outputs one by one:
    a unitary prefix keeps it pure (psi <- K psi with the sparse Kronecker
    embedding), then a few channels and a measurement turn it into a rank-r
    factored operator whose elements the oracle evaluates directly."""
    rng = S.rng_for(5000 + n)
    N = 1 << n
    psi = S.haar_state_vector(rng, N)
    unitary = [op for op in S.sweep(n) if op["kind"] == "unitary"]
    if n > 14:
        unitary = unitary[:: 3]
    channels = [S.op_depolarize(1, 0.1), S.op_ampdamp(n - 1, 0.05), S.op_depolarize(n - 3, 0.05)]
    tail = [S.op_unitary(S.haar_unitary(rng, 4), [2, n - 2]), S.op_unitary(S.haar_unitary(rng, 2), [n - 1])]
    h = _handle(n, dtype, 5)
    try:
        ok.orkan_init_state(h, ok.ORKAN_INIT_PURE, psi)
        vecs = [psi]
        for op in unitary:
            ok.orkan_apply_unitary(h, op["qubits"], op["matrix"])
            vecs = D.apply_kraus_to_factors(vecs, [op["matrix"]], op["qubits"], n)
        rows, cols = _sample_idx(rng, N, 4000)
        _assert_close(ok.orkan_get_elements(h, rows, cols), D.factored_elements(vecs, rows, cols), dtype,
                      "unitary sweep", rel=REL_BIG[dtype])
        for op in channels:
            circuit.apply_op(h, op)
            kr = D.depolarizing_kraus(op["p"]) if op["kind"] == "depolarize" else D.amplitude_damping_kraus(op["gamma"])
            vecs = D.apply_kraus_to_factors(vecs, kr, op["qubits"], n)
        q = 3
        p0 = sum(np.sum(np.abs(v[(np.arange(N) >> q) & 1 == 0]) ** 2) for v in vecs)
        p1 = sum(np.sum(np.abs(v[(np.arange(N) >> q) & 1 == 1]) ** 2) for v in vecs)
        u = 0.37
        assert abs(u - p0 / (p0 + p1)) > 1e-4
        b, pb = ok.orkan_measure(h, q, u)
        assert b == (0 if u * (p0 + p1) < p0 else 1)
        assert abs(pb - (p1 if b else p0) / (p0 + p1)) <= TOL[dtype] * 10
        vecs = D.apply_kraus_to_factors(vecs, [D.projector(b) / np.sqrt(p1 if b else p0)], [q], n)
        for op in tail:
            ok.orkan_apply_unitary(h, op["qubits"], op["matrix"])
            vecs = D.apply_kraus_to_factors(vecs, [op["matrix"]], op["qubits"], n)
        rows, cols = _sample_idx(rng, N, 4000)
        _assert_close(ok.orkan_get_elements(h, rows, cols), D.factored_elements(vecs, rows, cols), dtype,
                      "channels + measurement", rel=REL_BIG[dtype])
        assert abs(ok.orkan_trace(h) - 1.0) <= TOL[dtype] * 10
        for s in ("Z" * n, "X" + "I" * (n - 1), "IY" + "Z" * (n - 2)):
            x = sum((ord(c) in (88, 89)) << l for l, c in enumerate(s))
            # tr(P H) on the factored form, evaluated element by element by the oracle
            idx = np.arange(N)
            ph = np.ones(N, dtype=np.complex128)
            for l, c in enumerate(s):
                bit = (idx >> l) & 1
                if c == "Z":
                    ph *= np.where(bit == 1, -1, 1)
                elif c == "Y":
                    ph *= np.where(bit == 1, 1j, -1j)
            ref = np.sum(ph * D.factored_elements(vecs, idx ^ x, idx)).real
            assert abs(ok.orkan_expect_pauli(h, s) - ref) <= TOL[dtype] * 10 * max(abs(ref), 1e-3), s
    finally:
        ok.orkan_free(h)


# ------------------------------------------------------------------ autotuner
def test_autotune_choice_is_valid_cached_and_exact():
    m, f = ok.orkan_autotune(8, ok.ORKAN_DF64)
    assert 3 <= m <= 5 and 1 <= f <= 16
    assert ok.orkan_autotune(8, ok.ORKAN_DF64) == (m, f)        # cached for the process
    rng = S.rng_for(6000)
    n = 8
    psi = S.haar_state_vector(rng, 1 << n)
    ops = S.brickwork(n, 3, seed=6001)
    ref, _ = D.run_circuit(np.outer(psi, psi.conj()), ops)
    h = _handle(n, "df64", m, f, True)
    try:
        ok.orkan_init_state(h, ok.ORKAN_INIT_PURE, psi)
        circuit.run_circuit(h, ops)
        _assert_close(ok.orkan_to_dense(h), ref, "df64", "brickwork with autotuned settings")
    finally:
        ok.orkan_free(h)


# ------------------------------------------------------------------ native (monomial) gates
_S = np.diag([1, 1j]).astype(np.complex128)
_CNOT = np.eye(4, dtype=np.complex128)[[0, 3, 2, 1]]      # control = index bit 0
_CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)
_SWAP = np.eye(4, dtype=np.complex128)[[0, 2, 1, 3]]
_ISWAP = np.array([[1, 0, 0, 0], [0, 0, 1j, 0], [0, 1j, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
@pytest.mark.parametrize("picture", ["schrodinger", "heisenberg"])
def test_monomial_gates(dtype, picture):
    """X, Y, Z, S, S^dagger, CNOT, CZ, SWAP, iSWAP are permutations with
    quarter-turn phases (Sec. II-B native gates): applied without arithmetic,
    so native FP64 reproduces the oracle bit for bit."""
    n, m = 9, 3
    rng = S.rng_for(6500)
    H0 = S.random_hermitian(rng, 1 << n)
    gates1 = [D.X, D.Y, D.Z, _S, _S.conj().T]
    gates2 = [_CNOT, _CZ, _SWAP, _ISWAP]
    h = _handle(n, dtype, m, fusion=4, compose=False)
    try:
        for q in (0, 2, 3, 8):
            for U in gates1:
                ops = [S.op_unitary(U, [q])]
                _check_ops(h, H0, ops, dtype, picture, exact=(dtype == "c128"))
        for pair in ((0, 1), (1, 0), (2, 7), (8, 3), (5, 6)):
            for U in gates2:
                _check_ops(h, H0, [S.op_unitary(U, list(pair))], dtype, picture, exact=(dtype == "c128"))
        # fused runs mixing monomial and dense ops
        mix = [S.op_unitary(D.X, [4]), S.op_unitary(_CNOT, [4, 7]), S.op_unitary(S.haar_unitary(rng, 2), [4]),
               S.op_unitary(_ISWAP, [7, 8]), S.op_depolarize(8, 0.1), S.op_unitary(D.Y, [1])]
        _check_ops(h, H0, mix, dtype, picture, exact=False)
    finally:
        ok.orkan_free(h)


def _check_ops(h, H0, ops, dtype, picture, exact):
    ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, H0)
    if picture == "heisenberg":
        ok.orkan_set_picture(h, ok.ORKAN_OBSERVABLE)
    circuit.run_circuit(h, ops, picture)
    ref, _ = D.run_circuit(H0, ops, picture)
    got = ok.orkan_to_dense(h)
    if exact:
        assert np.array_equal(got, ref), [o["qubits"] for o in ops]
    else:
        _assert_close(got, ref, dtype, str([o["qubits"] for o in ops]))


# ------------------------------------------------------------------ captured circuits
@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
def test_graph_capture_replay(dtype):
    n = 9
    rng = S.rng_for(6600)
    rho0 = S.ginibre_state(rng, 1 << n)
    ops = S.random_mixed_circuit(rng, n, 40, with_measure=False)
    h1, h2 = _handle(n, dtype, 5), _handle(n, dtype, 5)
    try:
        ok.orkan_init_state(h1, ok.ORKAN_INIT_DENSE, rho0)
        ok.orkan_init_state(h2, ok.ORKAN_INIT_DENSE, rho0)
        ok.orkan_sync(h1)
        ok.orkan_capture_begin(h1)
        circuit.run_circuit(h1, ops)
        with pytest.raises(ok.OrkanError):
            ok.orkan_trace(h1)                     # blocking calls are refused while recording
        g = ok.orkan_capture_end(h1)
        assert np.array_equal(ok.orkan_to_dense(h1), ok.orkan_to_dense(h2))   # recording runs nothing
        ok.orkan_graph_launch(h1, g)
        ok.orkan_graph_launch(h1, g)
        circuit.run_circuit(h2, ops)
        circuit.run_circuit(h2, ops)
        assert np.array_equal(ok.orkan_to_dense(h1), ok.orkan_to_dense(h2))
        ref, _ = D.run_circuit(rho0, ops + ops)
        _assert_close(ok.orkan_to_dense(h1), ref, dtype, "replayed circuit")
        ok.orkan_graph_free(g)
    finally:
        ok.orkan_free(h1)
        ok.orkan_free(h2)


# ------------------------------------------------------------------ one-call circuits
@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
def test_native_circuit_runner_matches_per_op_calls(dtype):
    w = S.config0(n=7, depth=80)
    for picture in ("schrodinger", "heisenberg"):
        hs = [_handle(7, dtype, 5), _handle(7, dtype, 5)]
        try:
            for h in hs:
                ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, w["rho"])
                if picture == "heisenberg":
                    ok.orkan_set_picture(h, ok.ORKAN_OBSERVABLE)
            ops = w["ops"] if picture == "schrodinger" else [o for o in w["ops"] if o["kind"] != "measure"]
            r1 = circuit.run_circuit(hs[0], ops, picture, native=True)
            r2 = circuit.run_circuit(hs[1], ops, picture, native=False)
            assert r1 == r2
            assert np.array_equal(ok.orkan_to_dense(hs[0]), ok.orkan_to_dense(hs[1]))
        finally:
            for h in hs:
                ok.orkan_free(h)
