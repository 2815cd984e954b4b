"""Qubit relabelling: the logical operator never changes.

A relabelled handle must give the oracle's results through every call --
operations, measurements (same outcomes), Pauli expectations, elements,
dense export, tiled export, the packed copy, tr(rho O) between handles with
different labels, and captured graphs.  The automatic planner must move a
circuit's hot qubits into the tile and cut the number of passes.
"""
import numpy as np
import pytest

from oracle import dense as D
from oracle import packed as PK
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


def _close(got, ref, dtype, what=""):
    err = float(np.max(np.abs(got - ref)))
    assert err <= _tol(dtype, ref), f"{what}: {err:.3e}"


@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
@pytest.mark.parametrize("picture", ["schrodinger", "heisenberg"])
def test_relabelled_handle_matches_the_oracle(dtype, picture):
    n, m = 9, 3
    rng = S.rng_for(9000)
    N = 1 << n
    H0 = S.ginibre_state(rng, N) if picture == "schrodinger" else S.random_hermitian(rng, N)
    ops = S.random_mixed_circuit(rng, n, 60, with_measure=(picture == "schrodinger"))
    perm = [int(x) for x in rng.permutation(n)]
    h = ok.orkan_alloc(n, DT[dtype], m)
    try:
        ok.orkan_set_fusion(h, 8, True)
        ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, H0)
        if picture == "heisenberg":
            ok.orkan_set_picture(h, ok.ORKAN_OBSERVABLE)
        ok.orkan_relabel(h, perm)
        assert ok.orkan_get_labels(h, n) == perm
        _close(ok.orkan_to_dense(h), H0, dtype, "after relabel")
        recs = circuit.run_circuit(h, ops, picture)
        ref, ref_recs = D.run_circuit(H0, ops, picture)
        if picture == "schrodinger":
            assert [r[0] for r in recs] == [r[0] for r in ref_recs]
        _close(ok.orkan_to_dense(h), ref, dtype, "circuit")
        rows, cols = rng.integers(0, N, 300), rng.integers(0, N, 300)
        _close(ok.orkan_get_elements(h, rows, cols), ref[rows, cols], dtype, "elements")
        for s in S.random_pauli_strings(rng, n, 8):
            got = ok.orkan_expect_pauli(h, s)
            assert abs(got - D.expect_pauli(ref, s).real) <= 10 * _tol(dtype, ref) * N, s
        assert abs(ok.orkan_trace(h) - np.trace(ref)) <= 10 * _tol(dtype, ref) * N
        assert ok.orkan_get_labels(h, n) == perm
    finally:
        ok.orkan_free(h)


@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
def test_auto_relabel_moves_hot_qubits_into_the_tile(dtype):
    """A circuit on the three highest qubits: the planner swaps them below
    m = 3 and the circuit runs in fewer passes, with the oracle's result."""
    n, m = 10, 3
    rng = S.rng_for(9100)
    H0 = S.ginibre_state(rng, 1 << n)
    hot = [7, 8, 9]
    ops = []
    for layer in range(12):
        for q in hot:
            ops.append(S.op_unitary(S.haar_unitary(rng, 2), [q]))
        a, b = hot[layer % 2], hot[layer % 2 + 1]
        ops.append(S.op_unitary(S.haar_unitary(rng, 4), [a, b]))
        ops.append(S.op_depolarize(hot[layer % 3], 0.02))
    ref, _ = D.run_circuit(H0, ops)
    passes = {}
    for mode in (0, 1):
        h = ok.orkan_alloc(n, DT[dtype], m)
        try:
            ok.orkan_set_fusion(h, 16, True)
            ok.orkan_set_relabel(h, mode)
            ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, H0)
            p0 = ok.orkan_stats(h)["passes"]
            circuit.run_circuit(h, ops)
            ok.orkan_flush(h)
            passes[mode] = ok.orkan_stats(h)["passes"] - p0
            labels = ok.orkan_get_labels(h, n)
            if mode == 1:
                assert sorted(labels[q] for q in hot) == [0, 1, 2], labels
            else:
                assert labels == list(range(n))
            _close(ok.orkan_to_dense(h), ref, dtype, f"mode {mode}")
        finally:
            ok.orkan_free(h)
    assert passes[1] < passes[0], passes


def test_auto_relabel_leaves_uniform_circuits_alone():
    n, m = 9, 3
    ops = S.brickwork(n, 4)
    h = ok.orkan_alloc(n, DT["df64"], m)
    try:
        ok.orkan_set_relabel(h, 1)
        ok.orkan_init_state(h, ok.ORKAN_INIT_MAXMIXED)
        circuit.run_circuit(h, ops)
        assert ok.orkan_get_labels(h, n) == list(range(n))
    finally:
        ok.orkan_free(h)


@pytest.mark.parametrize("dtype", ["c128", "df64"])
def test_expect_between_differently_labelled_handles(dtype):
    n, m = 8, 3
    rng = S.rng_for(9200)
    rho0 = S.ginibre_state(rng, 1 << n)
    strings, coeffs = S.random_pauli_sum(rng, n, 16)
    O0 = D.pauli_sum(strings, coeffs)
    hr = ok.orkan_alloc(n, DT[dtype], m)
    ho = ok.orkan_alloc(n, DT[dtype], m)
    try:
        ok.orkan_init_state(hr, ok.ORKAN_INIT_DENSE, rho0)
        ok.orkan_init_observable(ho, strings, coeffs)
        ok.orkan_relabel(hr, [int(x) for x in rng.permutation(n)])
        ok.orkan_relabel(ho, [int(x) for x in rng.permutation(n)])
        got = ok.orkan_expect(hr, ho)
        ref = np.trace(rho0 @ O0).real
        assert abs(got - ref) <= 1e-11 * max(1.0, abs(ref))
        assert ok.orkan_get_labels(ho, n) == ok.orkan_get_labels(hr, n)
    finally:
        ok.orkan_free(hr)
        ok.orkan_free(ho)


def test_store_tiled_and_packed_copy_are_logical():
    """Exports hold the logical operator (bit for bit after permutations)."""
    torch = pytest.importorskip("torch")
    n, m = 7, 3
    rng = S.rng_for(9300)
    H0 = S.random_hermitian(rng, 1 << n)
    h = ok.orkan_alloc(n, DT["c128"], m)
    try:
        ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, H0)
        ok.orkan_relabel(h, [3, 6, 0, 5, 1, 2, 4])
        buf = np.empty(ok.orkan_bytes(n, DT["c128"], m), dtype=np.uint8)
        ok.orkan_store_tiled(h, buf)
        assert np.array_equal(buf.view(np.complex128), T.to_tiled(H0, m))
        assert ok.orkan_get_labels(h, n) == list(range(n))
        ok.orkan_relabel(h, [6, 5, 4, 3, 2, 1, 0])
        pk = torch.empty(ok.orkan_packed_bytes(n, DT["c128"]), dtype=torch.uint8, device="cuda")
        ok.orkan_set_stream(h, torch.cuda.current_stream().cuda_stream)
        ok.orkan_packed_from_tiled(h, pk.data_ptr())
        torch.cuda.current_stream().synchronize()
        assert np.array_equal(pk.cpu().numpy().view(np.complex128), PK.to_packed(H0))
    finally:
        ok.orkan_free(h)


def test_graph_replay_needs_the_captured_labels():
    n, m = 8, 3
    rng = S.rng_for(9400)
    H0 = S.ginibre_state(rng, 1 << n)
    ops = [S.op_unitary(S.haar_unitary(rng, 2), [q]) for q in range(n)]
    ops += [S.op_unitary(S.haar_unitary(rng, 4), [6, 7]), S.op_depolarize(7, 0.05)]
    perm = [4, 6, 2, 0, 1, 7, 5, 3]
    h = ok.orkan_alloc(n, DT["df64"], m)
    try:
        ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, H0)
        ok.orkan_capture_begin(h)
        ok.orkan_relabel(h, perm)           # recorded: the graph relabels, then runs the circuit
        circuit.run_circuit(h, ops)
        g = ok.orkan_capture_end(h)
        try:
            assert ok.orkan_get_labels(h, n) == list(range(n))   # recording ran nothing
            ok.orkan_relabel(h, perm)
            with pytest.raises(ok.OrkanError):
                ok.orkan_graph_launch(h, g)    # the graph starts from the identity labels
            ok.orkan_relabel(h, list(range(n)))
            ok.orkan_graph_launch(h, g)
            assert ok.orkan_get_labels(h, n) == perm
            ref, _ = D.run_circuit(H0, ops)
            _close(ok.orkan_to_dense(h), ref, "df64", "graph")
        finally:
            ok.orkan_graph_free(g)
    finally:
        ok.orkan_free(h)


def test_relabel_rejects_bad_maps():
    n = 5
    h = ok.orkan_alloc(n, DT["c128"], 3)
    try:
        ok.orkan_init_state(h, ok.ORKAN_INIT_MAXMIXED)
        for bad in ([0, 1, 2, 3, 3], [0, 1, 2, 3, 5], [-1, 0, 1, 2, 3]):
            with pytest.raises(ok.OrkanError):
                ok.orkan_relabel(h, bad)
            assert ok.orkan_get_labels(h, n) == list(range(n))
        with pytest.raises(ok.OrkanError):
            ok.orkan_set_relabel(h, 2)
    finally:
        ok.orkan_free(h)
