"""Tensor-core passes (orkan_set_tensor): runs of in-tile single-Kraus ops
composed into one 32 x 32 block and applied as L T L^dagger to every stored
tile with tcgen05 MMAs (complex64, m = 5), against the oracle and against the
CUDA-core passes of the same circuit.

Covers: one- and two-qubit Haar unitaries, monomial gates and a one-operator
Kraus map inside the tile; both pictures; a run longer than a fused pass
(one launch for 40 ops); a run ended by a cross-tile op; a padded operator
(n < m); a partial last work item (the stored tile count is not a multiple
of four); and graph capture of the pass.
"""
import numpy as np
import pytest

from oracle import dense as D
from workloads import synth as S

pytestmark = pytest.mark.gpu

ok = pytest.importorskip("paper_2604_15765_gb300.orkan")
from paper_2604_15765_gb300 import circuit  # noqa: E402

TOL = 1e-5


def _intile(rng, n, count):
    lo = min(n, 5)
    ops = []
    for i in range(count):
        c = i % 5
        if c in (0, 3) or lo == 1:
            ops.append(S.op_unitary(S.haar_unitary(rng, 2), [int(rng.integers(lo))]))
        elif c == 1:
            a, b = rng.choice(lo, size=2, replace=False)
            ops.append(S.op_unitary(S.haar_unitary(rng, 4), [int(a), int(b)]))
        elif c == 2:
            a, b = rng.choice(lo, size=2, replace=False)
            ops.append(S.op_unitary(np.eye(4, dtype=np.complex128)[[0, 1, 3, 2]], [int(a), int(b)]))   # CNOT
        else:
            a, b = rng.choice(lo, size=2, replace=False)
            K = np.sqrt(0.9) * S.haar_unitary(rng, 4)                                            # one Kraus operator
            ops.append(S.op_kraus([K], [int(a), int(b)]))
    return ops


def _run(n, ops, mode, picture="schrodinger", H0=None, seed=0):
    h = ok.orkan_alloc(n, ok.ORKAN_C64, 5)
    try:
        ok.orkan_set_tensor(h, mode)
        if picture == "schrodinger":
            ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, H0)
        else:
            ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, H0)
            ok.orkan_set_picture(h, ok.ORKAN_OBSERVABLE)
        p0 = ok.orkan_stats(h)["passes"]
        circuit.run_circuit(h, ops, picture)
        ok.orkan_sync(h)
        return ok.orkan_to_dense(h), ok.orkan_stats(h)["passes"] - p0
    finally:
        ok.orkan_free(h)


@pytest.mark.parametrize("n", [3, 5, 7, 8, 10])
@pytest.mark.parametrize("picture", ["schrodinger", "heisenberg"])
def test_tensor_pass_matches_oracle_and_cuda_cores(n, picture):
    rng = S.rng_for(6000 + 10 * n + (picture == "heisenberg"))
    H0 = S.ginibre_state(rng, 1 << n) if picture == "schrodinger" else S.random_hermitian(rng, 1 << n)
    ops = _intile(rng, n, 12)
    ref, _ = D.run_circuit(H0, ops, picture)
    scale = max(1.0, float(np.max(np.abs(ref))))
    tc, passes = _run(n, ops, 2, picture, H0)
    cc, _ = _run(n, ops, 0, picture, H0)
    assert passes == 1
    assert np.max(np.abs(tc - ref)) <= TOL * scale
    assert np.max(np.abs(tc - cc)) <= TOL * scale


def test_long_run_is_one_tensor_pass_and_a_cross_tile_op_ends_it():
    n = 9
    rng = S.rng_for(6100)
    rho = S.ginibre_state(rng, 1 << n)
    ops = _intile(rng, n, 40) + [S.op_unitary(S.haar_unitary(rng, 4), [1, 8])] + _intile(rng, n, 7)
    ref, _ = D.run_circuit(rho, ops)
    got, passes = _run(n, ops, 1, "schrodinger", rho)
    # the 40 in-tile ops as one tensor-core pass; the cross-tile op then opens an
    # ordinary fused pass that takes the last 7 ops with it
    assert passes == 2
    assert np.max(np.abs(got - ref)) <= TOL


def test_auto_mode_leaves_short_runs_on_cuda_cores():
    n = 8
    rng = S.rng_for(6200)
    rho = S.ginibre_state(rng, 1 << n)
    ops = [S.op_unitary(S.haar_unitary(rng, 2), [q]) for q in (0, 2, 4)]   # three single-qubit ops
    a, _ = _run(n, ops, 1, "schrodinger", rho)
    b, _ = _run(n, ops, 0, "schrodinger", rho)
    assert np.array_equal(a, b)


def test_captured_tensor_pass_replays():
    n = 8
    rng = S.rng_for(6300)
    rho = S.ginibre_state(rng, 1 << n)
    ops = _intile(rng, n, 10)
    ref, _ = D.run_circuit(rho, ops + ops)
    stream = __import__("torch").cuda.Stream()
    h = ok.orkan_alloc(n, ok.ORKAN_C64, 5)
    try:
        ok.orkan_set_stream(h, stream.cuda_stream)
        ok.orkan_set_tensor(h, 2)
        ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, rho)
        ok.orkan_capture_begin(h)
        circuit.run_circuit(h, ops)
        g = ok.orkan_capture_end(h)
        try:
            ok.orkan_graph_launch(h, g)
            ok.orkan_graph_launch(h, g)
        finally:
            ok.orkan_graph_free(g)
        ok.orkan_sync(h)
        assert np.max(np.abs(ok.orkan_to_dense(h) - ref)) <= TOL
    finally:
        ok.orkan_free(h)


@pytest.mark.parametrize("picture", ["schrodinger", "heisenberg"])
def test_three_qubit_ops_join_the_tensor_pass(picture):
    """In-tile three-qubit single-Kraus ops (a Haar unitary, a Toffoli) join
    the composed block instead of running the block-update kernel on their
    own; the run is one pass and matches the oracle and the CUDA-core path."""
    n = 8
    rng = S.rng_for(6400 + (picture == "heisenberg"))
    H0 = S.ginibre_state(rng, 1 << n) if picture == "schrodinger" else S.random_hermitian(rng, 1 << n)
    toffoli = np.eye(8, dtype=np.complex128)[[0, 1, 2, 7, 4, 5, 6, 3]]
    ops = _intile(rng, n, 4) + [S.op_unitary(S.haar_unitary(rng, 8), [4, 0, 2]),
                                S.op_unitary(toffoli, [1, 3, 0])] + _intile(rng, n, 3)
    ref, _ = D.run_circuit(H0, ops, picture)
    scale = max(1.0, float(np.max(np.abs(ref))))
    tc, passes = _run(n, ops, 1, picture, H0)
    cc, _ = _run(n, ops, 0, picture, H0)
    assert passes == 1
    assert np.max(np.abs(tc - ref)) <= TOL * scale
    assert np.max(np.abs(cc - ref)) <= TOL * scale


@pytest.mark.parametrize("compose", [True, False])
def test_long_run_ends_before_a_channel_on_its_last_qubit(compose):
    """A tensor-core run longer than a fused pass holds (here 20 dense in-tile
    unitaries) must leave as a tensor-core pass before a channel that cannot
    join it -- also when the channel would compose into the run's last
    single-qubit op (a regression: the merged run once became an ordinary
    pass of more than 16 ops)."""
    n = 6
    rng = S.rng_for(6500 + compose)
    rho = S.ginibre_state(rng, 1 << n)
    ops = []
    for _ in range(20):
        a, b = rng.choice(5, size=2, replace=False)
        ops.append(S.op_unitary(S.haar_unitary(rng, 4), [int(a), int(b)]))
    ops += [S.op_unitary(S.haar_unitary(rng, 2), [0]), S.op_unitary(S.haar_unitary(rng, 2), [1]),
            S.op_ampdamp(0, 0.3), S.op_depolarize(1, 0.1), S.op_unitary(S.haar_unitary(rng, 4), [2, 5])]
    ref, _ = D.run_circuit(rho, ops)
    h = ok.orkan_alloc(n, ok.ORKAN_C64, 5)
    try:
        ok.orkan_set_fusion(h, 8, compose)
        ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, rho)
        circuit.run_circuit(h, ops)
        ok.orkan_sync(h)
        assert np.max(np.abs(ok.orkan_to_dense(h) - ref)) <= TOL
    finally:
        ok.orkan_free(h)


def test_full_size_tensor_pass_matches_oracle_on_sampled_elements():
    """n = 13 (32,896 tiles, 269 MB): a 12-op in-tile run as one tensor-core
    pass, on 65,536 sampled elements and the diagonal, against the oracle's
    factored evaluation of Eq. (1) (the pure initial state stays a single
    factor under one-operator maps) and against the CUDA-core passes of the
    same run."""
    n = 13
    rng = S.rng_for(6600)
    psi = S.haar_state_vector(rng, 1 << n)
    ops = _intile(rng, n, 12)
    N = 1 << n
    rows = np.concatenate([rng.integers(0, N, 1 << 16), np.arange(N)])
    cols = np.concatenate([rng.integers(0, N, 1 << 16), np.arange(N)])
    vecs = [psi]
    for op in ops:
        mats = [op["matrix"]] if op["kind"] == "unitary" else op["mats"]
        vecs = D.apply_kraus_to_factors(vecs, mats, op["qubits"], n)
    ref = D.factored_elements(vecs, rows, cols)
    got = {}
    for mode in (2, 0):
        h = ok.orkan_alloc(n, ok.ORKAN_C64, 5)
        try:
            ok.orkan_set_tensor(h, mode)
            ok.orkan_init_state(h, ok.ORKAN_INIT_PURE, psi)
            p0 = ok.orkan_stats(h)["passes"]
            circuit.run_circuit(h, ops)
            ok.orkan_sync(h)
            if mode == 2:
                assert ok.orkan_stats(h)["passes"] - p0 == 1
            got[mode] = ok.orkan_get_elements(h, rows, cols)
        finally:
            ok.orkan_free(h)
    scale = max(float(np.max(np.abs(ref))), 1e-3)
    assert np.max(np.abs(got[2] - ref)) <= TOL * scale
    assert np.max(np.abs(got[2] - got[0])) <= TOL * scale
