"""GPU parity of three-qubit operations (Algorithm 1 with k = 3) against the oracle.

Covers every placement class of the three targets relative to the tile size
(all in-tile, one, two or three cross-tile qubits, so blocks spanning 1 to 64
tiles), the caller's qubit order, padded single-tile operators (n < m),
unitaries, Kraus sets up to the 16-operator limit, monomial gates (bit-exact),
both pictures, all three storage types, mixing with fused passes, graph
replay, and the full-size bench geometry on sampled elements.
Tolerances as in test_gpu_parity: 1e-12 * max(1, max|H|) for c128 / df64,
1e-5 * max|H| for c64.
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
DT = {"c128": 0, "c64": 1, "df64": 2}


def _tol(dtype, ref):
    scale = float(np.max(np.abs(ref)))
    return TOL[dtype] * (scale if dtype == "c64" else max(1.0, scale))


def _close(got, ref, dtype, what):
    err = float(np.max(np.abs(got - ref)))
    assert err <= _tol(dtype, ref), f"{what}: max|delta| = {err:.3e} > {_tol(dtype, ref):.1e}"


def _toffoli():
    T3 = np.zeros((8, 8), dtype=np.complex128)
    for b in range(8):
        T3[b ^ (4 if (b & 3) == 3 else 0), b] = 1
    return T3


def _fredkin():
    """Control on index bit 0, swaps the qubits of bits 1 and 2."""
    F = np.zeros((8, 8), dtype=np.complex128)
    for b in range(8):
        t = b
        if b & 1:
            t = (b & 1) | (((b >> 2) & 1) << 1) | (((b >> 1) & 1) << 2)
        F[t, b] = 1
    return F


CCZ = np.diag([1, 1, 1, 1, 1, 1, 1, -1]).astype(np.complex128)


def _random_monomial(rng):
    p = rng.permutation(8)
    ph = (1j) ** rng.integers(0, 4, 8)
    V = np.zeros((8, 8), dtype=np.complex128)
    V[np.arange(8), p] = ph
    return V


def _triples(n, m, rng, count):
    """Ordered target triples covering 0..3 cross-tile qubits, adjacent and
    far placements, and unsorted caller orders."""
    allt = list(itertools.permutations(range(n), 3))
    if len(allt) <= count:
        return allt
    by_high = {}
    for t in allt:
        by_high.setdefault(sum(q >= m for q in t), []).append(t)
    pick = [(0, 1, 2), (n - 1, n - 2, n - 3), (0, n // 2, n - 1), (n - 1, 0, n // 2)]
    for hi in sorted(by_high):
        group = by_high[hi]
        for i in rng.choice(len(group), min(3, len(group)), replace=False):
            pick.append(group[int(i)])
    return list(dict.fromkeys(pick))


def _init(h, H0, picture):
    ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, H0)
    if picture == "heisenberg":
        ok.orkan_set_picture(h, ok.ORKAN_OBSERVABLE)


K3_CASES = [(3, 5), (4, 5), (3, 3), (5, 3), (6, 3), (6, 5), (7, 3), (8, 4), (9, 3), (10, 5)]


@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
@pytest.mark.parametrize("picture", ["schrodinger", "heisenberg"])
@pytest.mark.parametrize("n,m", K3_CASES)
def test_k3_unitary_placements(n, m, dtype, picture):
    rng = S.rng_for(7000 + 17 * n + m)
    N = 1 << n
    H0 = S.ginibre_state(rng, N) if picture == "schrodinger" else S.random_hermitian(rng, N)
    h = ok.orkan_alloc(n, DT[dtype], m)
    try:
        for t in _triples(n, m, rng, 40):
            U = S.haar_unitary(rng, 8)
            _init(h, H0, picture)
            ok.orkan_apply_unitary(h, list(t), U)
            ref = D.apply_unitary(H0, U, list(t), picture)
            _close(ok.orkan_to_dense(h), ref, dtype, f"U3 on {t}")
    finally:
        ok.orkan_free(h)


def _kraus_set(rng, r):
    """r operators of a random 3-qubit channel (blocks of a Haar isometry),
    scaled below trace preservation so that the map is trace non-increasing."""
    V = S.haar_unitary(rng, 8 * r)
    return [0.9 * V[8 * a:8 * (a + 1), :8] for a in range(r)]


@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
@pytest.mark.parametrize("picture", ["schrodinger", "heisenberg"])
@pytest.mark.parametrize("r", [2, 4, 16])
def test_k3_kraus(r, dtype, picture):
    n, m = 7, 3
    rng = S.rng_for(7100 + r)
    N = 1 << n
    H0 = S.ginibre_state(rng, N) if picture == "schrodinger" else S.random_hermitian(rng, N)
    h = ok.orkan_alloc(n, DT[dtype], m)
    try:
        for t in [(0, 1, 2), (6, 3, 4), (2, 5, 0), (1, 6, 3)]:
            ks = _kraus_set(rng, r)
            _init(h, H0, picture)
            ok.orkan_apply_kraus(h, list(t), np.array(ks))
            ref = D.apply_kraus(H0, ks, list(t), picture)
            _close(ok.orkan_to_dense(h), ref, dtype, f"Kraus r={r} on {t}")
    finally:
        ok.orkan_free(h)


@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
@pytest.mark.parametrize("picture", ["schrodinger", "heisenberg"])
def test_k3_monomial_gates_are_exact(dtype, picture):
    """Toffoli, CCZ, Fredkin and a random monomial with quarter-turn phases
    permute the block without arithmetic: the result equals the oracle's map
    of the operator as stored, bit for bit, in every storage type."""
    n, m = 8, 3
    rng = S.rng_for(7200)
    H0 = S.random_hermitian(rng, 1 << n)
    h = ok.orkan_alloc(n, DT[dtype], m)
    try:
        for t in [(0, 1, 2), (7, 6, 5), (2, 6, 4), (5, 0, 7), (3, 1, 6)]:
            for U in (_toffoli(), CCZ, _fredkin(), _random_monomial(rng)):
                _init(h, H0, picture)
                before = ok.orkan_to_dense(h)
                ok.orkan_apply_unitary(h, list(t), U)
                ref = D.apply_unitary(before, U, list(t), picture)
                assert np.array_equal(ok.orkan_to_dense(h), ref), t
    finally:
        ok.orkan_free(h)


@pytest.mark.parametrize("dtype", ["c128", "df64"])
def test_k3_keeps_diagonal_tiles_hermitian(dtype):
    """Diagonal tiles store both halves; after a three-qubit op every upper
    element is exactly the conjugate of its lower partner (one writer per
    mirror pair)."""
    n, m = 7, 3
    M = 1 << m
    rng = S.rng_for(7300)
    h = ok.orkan_alloc(n, DT[dtype], m)
    try:
        ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, S.ginibre_state(rng, 1 << n))
        for t in [(0, 4, 6), (1, 2, 5)]:
            ok.orkan_apply_unitary(h, list(t), S.haar_unitary(rng, 8))
        raw = np.empty(ok.orkan_bytes(n, DT[dtype], m), dtype=np.uint8)
        ok.orkan_store_tiled(h, raw)
        vals = raw.view(np.float64 if dtype == "c128" else np.float32)
        vals = vals.reshape(-1, 2 if dtype == "c128" else 4)
        # element components: (re, im) for c128, (re.hi, im.hi, re.lo, im.lo) for df64
        re_c, im_c = ([0], [1]) if dtype == "c128" else ([0, 2], [1, 3])
        nt = (1 << n) // M
        off_diag = ~np.eye(M, dtype=bool)
        for ti in range(nt):
            off = (ti * (ti + 1) // 2 + ti) * M * M
            tile = vals[off:off + M * M].reshape(M, M, -1)
            up = tile.transpose(1, 0, 2)
            # off the global diagonal: the upper half mirrors the lower exactly
            assert np.array_equal(tile[off_diag][:, re_c], up[off_diag][:, re_c])     # real parts
            assert np.array_equal(tile[off_diag][:, im_c], -up[off_diag][:, im_c])    # imaginary parts
            # on it the imaginary part is the rounding residue of a real value
            assert np.max(np.abs(tile[~off_diag][:, im_c])) <= 1e-15
    finally:
        ok.orkan_free(h)


@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
@pytest.mark.parametrize("picture", ["schrodinger", "heisenberg"])
def test_k3_in_fused_circuits_and_native_runner(dtype, picture):
    """Three-qubit ops between fused one- and two-qubit runs, through the
    one-call circuit runner and through per-op calls."""
    n, m = 9, 4
    rng = S.rng_for(7400)
    H0 = S.ginibre_state(rng, 1 << n) if picture == "schrodinger" else S.random_hermitian(rng, 1 << n)
    ops = []
    for layer in range(3):
        for q in range(n):
            ops.append(S.op_unitary(S.haar_unitary(rng, 2), [q]))
        ops.append(S.op_unitary(S.haar_unitary(rng, 8), [layer, 5 + layer, 8 - layer]))
        ops.append(S.op_unitary(S.haar_unitary(rng, 4), [2, 6]))
        ops.append(S.op_unitary(_toffoli(), [8, layer, 4]))
        ops.append(S.op_kraus(_kraus_set(rng, 3), [7, 1, 3]))
        ops.append(S.op_depolarize(layer + 1, 0.05))
    ref, _ = D.run_circuit(H0, ops, picture)
    for native in (True, False):
        h = ok.orkan_alloc(n, DT[dtype], m)
        try:
            ok.orkan_set_fusion(h, 8, True)
            _init(h, H0, picture)
            circuit.run_circuit(h, ops, picture, native=native)
            _close(ok.orkan_to_dense(h), ref, dtype, f"native={native}")
        finally:
            ok.orkan_free(h)


def test_k3_graph_replay_matches_direct():
    n, m = 8, 3
    rng = S.rng_for(7500)
    H0 = S.ginibre_state(rng, 1 << n)
    ops = [S.op_unitary(S.haar_unitary(rng, 8), [0, 4, 7]), S.op_unitary(_toffoli(), [6, 1, 3]),
           S.op_unitary(S.haar_unitary(rng, 2), [5]), S.op_kraus(_kraus_set(rng, 2), [2, 3, 6])]
    h = ok.orkan_alloc(n, DT["df64"], m)
    try:
        ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, H0)
        circuit.run_circuit(h, ops)
        direct = ok.orkan_to_dense(h)
        ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, H0)
        ok.orkan_capture_begin(h)
        circuit.run_circuit(h, ops)
        g = ok.orkan_capture_end(h)
        try:
            ok.orkan_graph_launch(h, g)
            assert np.array_equal(ok.orkan_to_dense(h), direct)
        finally:
            ok.orkan_graph_free(g)
    finally:
        ok.orkan_free(h)


def test_k3_argument_errors():
    h = ok.orkan_alloc(5, DT["c128"], 5)
    try:
        with pytest.raises(RuntimeError):
            ok.orkan_apply_unitary(h, [0, 1, 1], np.eye(8))
        with pytest.raises(RuntimeError):
            ok.orkan_apply_unitary(h, [0, 1, 5], np.eye(8))
        with pytest.raises(RuntimeError):
            ok.orkan_apply_kraus(h, [0, 1, 2], np.array([np.eye(8) / 5.0] * 17))
    finally:
        ok.orkan_free(h)
    h2 = ok.orkan_alloc(2, DT["c128"], 5)
    try:
        with pytest.raises(RuntimeError):
            ok.orkan_apply_unitary(h2, [0, 1, 2], np.eye(8))
    finally:
        ok.orkan_free(h2)


@pytest.mark.parametrize("dtype", ["df64", "c128", "c64"])
def test_k3_full_size_sampled(dtype):
    """n = 14 at m = 5, the bench's geometry: three-qubit unitaries, a
    Toffoli and a Kraus set on pure-state factors, checked on sampled
    elements the oracle computes one by one."""
    n = 14
    N = 1 << n
    rng = S.rng_for(7600)
    psi = S.haar_state_vector(rng, N)
    h = ok.orkan_alloc(n, DT[dtype], 5)
    try:
        ok.orkan_init_state(h, ok.ORKAN_INIT_PURE, psi)
        vecs = [psi]
        for t, U in [((0, 7, 13), S.haar_unitary(rng, 8)), ((13, 12, 11), _toffoli()),
                     ((2, 3, 4), S.haar_unitary(rng, 8)), ((9, 1, 6), S.haar_unitary(rng, 8))]:
            ok.orkan_apply_unitary(h, list(t), U)
            vecs = D.apply_kraus_to_factors(vecs, [U], list(t), n)
        ks = _kraus_set(rng, 2)
        ok.orkan_apply_kraus(h, [10, 5, 12], np.array(ks))
        vecs = D.apply_kraus_to_factors(vecs, ks, [10, 5, 12], n)
        rows = np.concatenate([rng.integers(0, N, 3000), np.arange(0, N, 97)])
        cols = np.concatenate([rng.integers(0, N, 3000), np.arange(0, N, 97)])
        ref = D.factored_elements(vecs, rows, cols)
        got = ok.orkan_get_elements(h, rows, cols)
        # relative to the operator's scale, as for the other full-size checks
        tol = (1e-10 if dtype != "c64" else 1e-5) * float(np.max(np.abs(ref)))
        assert float(np.max(np.abs(got - ref))) <= tol
        assert abs(ok.orkan_trace(h) - 0.81) <= (1e-12 if dtype != "c64" else 1e-5)
    finally:
        ok.orkan_free(h)
