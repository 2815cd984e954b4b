"""Single-qubit ops held back and absorbed by the next dense two-qubit op on
their qubit (the planner's fold), against the oracle:

* a layered circuit (a single-qubit gate on every qubit, two-qubit gates on
  pairs, a channel on every qubit) in both pictures and all dtypes gives the
  oracle's operator with fewer FP64 / FP32 operations (the single-qubit gates
  run inside the two-qubit bodies);
* a held op is applied before any readout, measurement, projection or
  three-qubit op that follows it, and before a permutation gate (which does
  not absorb it);
* with fusion depth 1 (the plain path) nothing is held.
"""
import numpy as np
import pytest

from oracle import dense as D
from workloads import synth as S

pytestmark = pytest.mark.gpu

ok = pytest.importorskip("paper_2604_15765_gb300.orkan")
from paper_2604_15765_gb300 import circuit  # noqa: E402

TOL = {"c128": 1e-12, "df64": 1e-12, "c64": 1e-5}
DT = {"c128": ok.ORKAN_C128, "df64": ok.ORKAN_DF64, "c64": ok.ORKAN_C64}


@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
@pytest.mark.parametrize("picture", ["schrodinger", "heisenberg"])
def test_layered_circuit_matches_oracle(dtype, picture):
    n = 8
    rng = S.rng_for(7300 + len(dtype) + (picture == "heisenberg"))
    ops = S.brickwork(n, 3, seed=7301)
    H0 = S.ginibre_state(rng, 1 << n) if picture == "schrodinger" else S.random_hermitian(rng, 1 << n)
    ref, _ = D.run_circuit(H0, ops, picture)
    scale = max(1.0, float(np.max(np.abs(ref))))
    work = {}
    for fold in (True, False):
        h = ok.orkan_alloc(n, DT[dtype], 3)
        try:
            ok.orkan_set_fusion(h, 8, fold)      # composition (and the fold) on / off
            ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, H0)
            if picture == "heisenberg":
                ok.orkan_set_picture(h, ok.ORKAN_OBSERVABLE)
            ok.orkan_set_timing(h, True)
            ok.orkan_pass_work(h)
            circuit.run_circuit(h, ops, picture)
            ok.orkan_sync(h)
            work[fold] = ok.orkan_pass_work(h)[0]
            assert np.max(np.abs(ok.orkan_to_dense(h) - ref)) <= TOL[dtype] * scale * 10
        finally:
            ok.orkan_free(h)
    assert work[True] < 0.9 * work[False]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_held_op_is_applied_before_what_follows_it(dtype):
    n = 6
    rng = S.rng_for(7400)
    rho = S.ginibre_state(rng, 1 << n)
    u = S.haar_unitary(rng, 2)
    toffoli = np.eye(8, dtype=np.complex128)[[0, 1, 2, 7, 4, 5, 6, 3]]
    cnot = np.eye(4, dtype=np.complex128)[[0, 1, 3, 2]]
    cases = [
        [S.op_unitary(u, [2])],                                          # then a readout
        [S.op_unitary(u, [2]), S.op_measure(2, 0.4)],
        [S.op_unitary(u, [1]), S.op_project(1, 0)],
        [S.op_unitary(u, [0]), S.op_unitary(toffoli, [0, 4, 5])],
        [S.op_unitary(u, [3]), S.op_unitary(cnot, [3, 4])],
        [S.op_unitary(u, [3]), S.op_depolarize(3, 0.2), S.op_unitary(S.haar_unitary(rng, 4), [3, 5])],
    ]
    for ops in cases:
        ref, recs = D.run_circuit(rho, ops)
        h = ok.orkan_alloc(n, DT[dtype], 3)
        try:
            ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, rho)
            got_recs = circuit.run_circuit(h, ops)
            assert [b for b, _ in got_recs] == [b for b, _ in recs]
            for s in ("ZIYIXI", "IIZIII", "XXIIZZ"):
                assert abs(ok.orkan_expect_pauli(h, s) - D.expect_pauli(ref, s).real) <= TOL[dtype] * 10
            assert np.max(np.abs(ok.orkan_to_dense(h) - ref)) <= TOL[dtype] * 10
        finally:
            ok.orkan_free(h)


def test_plain_path_holds_nothing():
    n = 6
    rng = S.rng_for(7500)
    ops = S.brickwork(n, 2, seed=7501)
    h = ok.orkan_alloc(n, ok.ORKAN_C128, 3)
    try:
        ok.orkan_set_fusion(h, 1, False)
        ok.orkan_init_state(h, ok.ORKAN_INIT_MAXMIXED)
        circuit.run_circuit(h, ops)
        ok.orkan_sync(h)
        assert ok.orkan_stats(h)["passes"] == len(ops)
    finally:
        ok.orkan_free(h)
