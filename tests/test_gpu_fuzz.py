"""Randomised end-to-end parity: every op class mixed in random circuits, run
under random planner settings (tile size, fusion depth, composition,
automatic relabelling), storage types and pictures, against the oracle.

The settings and circuits are drawn from a fixed seed, so every case is
reproducible; the case id names its draw.
"""
import numpy as np
import pytest

from oracle import dense as D
from workloads import synth as S

pytestmark = pytest.mark.gpu

ok = pytest.importorskip("paper_2604_15765_gb300.orkan")
from paper_2604_15765_gb300 import circuit  # noqa: E402

TOL = {"c128": 1e-12, "df64": 1e-12, "c64": 2e-5}
DT = {"c128": 0, "c64": 1, "df64": 2}
TOFFOLI = np.eye(8, dtype=np.complex128)[[0, 1, 2, 7, 4, 5, 6, 3]]
CNOT = np.eye(4, dtype=np.complex128)[[0, 3, 2, 1]]


def _kraus(rng, d, r, scale):
    return [scale * (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) for _ in range(r)]


def _random_circuit(rng, n, depth, picture):
    ops = []
    for _ in range(depth):
        kind = rng.choice(["u1", "u2", "u3", "k1", "k2", "k3", "depol", "damp", "deph", "x", "cnot", "toffoli",
                           "measure"], p=[.18, .16, .06, .06, .05, .03, .08, .07, .05, .07, .07, .04, .08])
        q = [int(x) for x in rng.permutation(n)]
        if kind == "u1":
            ops.append(S.op_unitary(S.haar_unitary(rng, 2), q[:1]))
        elif kind == "u2" and n >= 2:
            ops.append(S.op_unitary(S.haar_unitary(rng, 4), q[:2]))
        elif kind == "u3" and n >= 3:
            ops.append(S.op_unitary(S.haar_unitary(rng, 8), q[:3]))
        elif kind == "k1":
            ops.append(S.op_kraus(_kraus(rng, 2, 3, 0.4), q[:1]))
        elif kind == "k2" and n >= 2:
            ops.append(S.op_kraus(_kraus(rng, 4, 2, 0.3), q[:2]))
        elif kind == "k3" and n >= 3:
            ops.append(S.op_kraus(_kraus(rng, 8, 2, 0.2), q[:3]))
        elif kind == "depol":
            ops.append(S.op_depolarize(q[0], float(rng.uniform(0, 0.2))))
        elif kind == "damp":
            ops.append(S.op_ampdamp(q[0], float(rng.uniform(0, 0.3))))
        elif kind == "deph":
            ops.append(S.op_dephase(q[0], float(rng.uniform(0, 0.3))))
        elif kind == "x":
            ops.append(S.op_unitary(D.X, q[:1]))
        elif kind == "cnot" and n >= 2:
            ops.append(S.op_unitary(CNOT, q[:2]))
        elif kind == "toffoli" and n >= 3:
            ops.append(S.op_unitary(TOFFOLI, q[:3]))
        elif kind == "measure":
            # projections keep the map linear in both pictures (Born sampling is covered elsewhere)
            ops.append(S.op_project(q[0], int(rng.integers(0, 2))))
    return ops


CASES = list(range(160))


@pytest.mark.parametrize("case", CASES)
def test_random_circuits_random_settings(case):
    rng = S.rng_for(11000 + case)
    n = int(rng.integers(3, 10))
    m = int(rng.choice([3, 4, 5]))
    dtype = str(rng.choice(["c128", "df64", "c64"]))
    picture = str(rng.choice(["schrodinger", "heisenberg"]))
    fusion = int(rng.choice([1, 2, 4, 8, 16]))
    compose = bool(rng.integers(0, 2))
    relabel = int(rng.integers(0, 2))
    native = bool(rng.integers(0, 2))
    N = 1 << n
    H0 = S.ginibre_state(rng, N) if picture == "schrodinger" else S.random_hermitian(rng, N)
    ops = _random_circuit(rng, n, int(rng.integers(10, 40)), picture)
    ref, _ = D.run_circuit(H0, ops, picture)
    h = ok.orkan_alloc(n, DT[dtype], m)
    try:
        ok.orkan_set_fusion(h, fusion, compose)
        ok.orkan_set_relabel(h, relabel)
        ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, H0)
        if picture == "heisenberg":
            ok.orkan_set_picture(h, ok.ORKAN_OBSERVABLE)
        if relabel and not native:
            ok.orkan_relabel(h, [int(x) for x in rng.permutation(n)])   # the per-op path has no planner
        circuit.run_circuit(h, ops, picture, native=native)
        got = ok.orkan_to_dense(h)
        scale = float(np.max(np.abs(ref)))
        tol = TOL[dtype] * (scale if dtype == "c64" else max(1.0, scale))
        err = float(np.max(np.abs(got - ref)))
        what = f"n={n} m={m} {dtype} {picture} fusion={fusion} compose={compose} relabel={relabel} native={native}"
        assert err <= tol, f"{what}: max|delta| {err:.3e} > {tol:.1e}"
        s = S.random_pauli_strings(rng, n, 1)[0]
        assert abs(ok.orkan_expect_pauli(h, s) - D.expect_pauli(ref, s).real) <= 50 * tol * N, what
    finally:
        ok.orkan_free(h)
