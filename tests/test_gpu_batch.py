"""Batched circuits (orkan_run_batch): many small operators' whole circuits
in one persistent launch per dtype, against the oracle.

* A batch mixing n = 4..9, all three dtypes, both pictures, every op class
  (1-, 2-, 3-qubit unitaries and Kraus sets, named channels, measurements,
  projections) and both readouts matches the dense oracle: final operators,
  measurement outcomes, Pauli expectations and <psi|O|psi>.  n <= 7 runs in
  shared memory on one CTA, n = 8, 9 on gangs of CTAs.
* A request gives the same bits alone and in a mix.
* A forced gang, a relabelled handle kept as it is, a zero-probability
  measurement and a gang that cannot assemble (ORKAN_ETIMEOUT, after which
  the context still works) behave as documented.
"""
import numpy as np
import pytest

from oracle import dense as D
from workloads import synth as S

pytestmark = pytest.mark.gpu

ok = pytest.importorskip("paper_2604_15765_gb300.orkan")
from paper_2604_15765_gb300 import circuit  # noqa: E402

TOL = {ok.ORKAN_C128: 1e-12, ok.ORKAN_DF64: 1e-12, ok.ORKAN_C64: 1e-5}
DTYPES = (ok.ORKAN_C128, ok.ORKAN_DF64, ok.ORKAN_C64)


def _kraus2(rng):
    """A two-qubit Kraus set: sqrt(1-p) U_a, sqrt(p) U_b."""
    p = 0.3
    return [np.sqrt(1 - p) * S.haar_unitary(rng, 4), np.sqrt(p) * S.haar_unitary(rng, 4)]


def _circuit(rng, n, depth, measure):
    ops = S.random_mixed_circuit(rng, n, depth, with_measure=measure)
    a, b, c = (int(x) for x in rng.choice(n, size=3, replace=False))
    ops.insert(3, S.op_unitary(S.haar_unitary(rng, 8), [a, b, c]))
    ops.insert(7, S.op_kraus(_kraus2(rng), [c, a]))
    ops.insert(9, S.op_dephase(b, 0.07))
    ops.insert(11, S.op_project(a, int(rng.integers(2))) if not measure else S.op_depolarize(c, 0.02))
    return ops


def _request(rng, n, dt, picture):
    h = ok.orkan_alloc(n, dt, 5)
    if picture == "schrodinger":
        psi0 = S.haar_state_vector(rng, 1 << n)
        ops = _circuit(rng, n, 20, True)
        req = {"h": h, "init": "pure", "psi0": psi0, "ops": ops, "paulis": S.random_pauli_strings(rng, n, 6)}
        H0 = np.outer(psi0, psi0.conj())
    else:
        terms, coeffs = S.random_pauli_sum(rng, n, 16)
        ops = _circuit(rng, n, 20, False)
        req = {"h": h, "init": "pauli_sum", "terms": terms, "coeffs": coeffs, "ops": ops,
               "paulis": S.random_pauli_strings(rng, n, 3), "psi": S.random_product_vector(rng, n)}
        H0 = D.pauli_sum(terms, coeffs)
    ref, recs = D.run_circuit(H0, ops, picture)
    return req, ref, recs, dt, picture


def _check(req, ref, recs, dt, picture, res):
    assert res["status"] == ok.ORKAN_OK
    scale = max(1.0, float(np.max(np.abs(ref))))
    got = ok.orkan_to_dense(req["h"])
    assert np.max(np.abs(got - ref)) <= TOL[dt] * scale * 10
    if picture == "schrodinger":
        assert res["outcomes"] == [b for b, _ in recs]
        for (_, pb), p in zip(recs, res["probs"]):
            assert p == pytest.approx(pb, abs=TOL[dt] * 10)
    want = [D.expect_pauli(ref, s).real for s in req["paulis"]]
    if req.get("psi") is not None:
        v = req["psi"]
        want.append(float(np.real(v.conj() @ ref @ v)))
    assert np.max(np.abs(res["out"] - np.array(want))) <= TOL[dt] * scale * 100


def test_mixed_batch_matches_the_oracle():
    rng = S.rng_for(5100)
    cases = []
    for n in range(4, 10):
        for j, dt in enumerate(DTYPES):
            cases.append(_request(rng, n, dt, "schrodinger" if (n + j) % 2 == 0 else "heisenberg"))
    try:
        res = circuit.run_batch([c[0] for c in cases])
        for c, r in zip(cases, res):
            _check(*c, r)
    finally:
        for c in cases:
            ok.orkan_free(c[0]["h"])


def test_largest_gangs_match_the_oracle():
    """The largest gangs, 64 CTAs (n = 10 in native FP64, automatic; n = 10
    in complex64, forced), and an automatic 17-CTA double-float gang (n = 10),
    each group's grid holding its gang whole, against the oracle."""
    rng = S.rng_for(5150)
    cases = [_request(rng, 10, ok.ORKAN_C128, "schrodinger"), _request(rng, 10, ok.ORKAN_C64, "heisenberg"),
             _request(rng, 10, ok.ORKAN_DF64, "schrodinger")]
    cases[1][0]["gang"] = 64
    try:
        res = circuit.run_batch([c[0] for c in cases])
        for c, r in zip(cases, res):
            _check(*c, r)
    finally:
        for c in cases:
            ok.orkan_free(c[0]["h"])


def test_request_is_bitwise_the_same_alone_and_in_a_mix():
    rng = S.rng_for(5200)
    reqs = [_request(rng, n, ok.ORKAN_C128, pic)[0]
            for n, pic in ((6, "schrodinger"), (8, "heisenberg"), (5, "schrodinger"), (9, "schrodinger"))]
    try:
        for target in (0, 1, 3):
            alone = circuit.run_batch([reqs[target]])[0]
            dense_alone = ok.orkan_to_dense(reqs[target]["h"])
            mix = circuit.run_batch(reqs)[target]
            assert np.array_equal(alone["out"], mix["out"])
            assert alone["outcomes"] == mix["outcomes"]
            assert np.array_equal(dense_alone, ok.orkan_to_dense(reqs[target]["h"]))
    finally:
        for r in reqs:
            ok.orkan_free(r["h"])


@pytest.mark.parametrize("dt", DTYPES)
def test_forced_gang_matches_one_cta(dt):
    rng = S.rng_for(5300 + dt)
    req, ref, recs, _, pic = _request(rng, 6, dt, "schrodinger")
    try:
        one = circuit.run_batch([dict(req, gang=1)])[0]
        d1 = ok.orkan_to_dense(req["h"])
        three = circuit.run_batch([dict(req, gang=3)])[0]
        _check(req, ref, recs, dt, pic, three)
        assert np.max(np.abs(ok.orkan_to_dense(req["h"]) - d1)) <= TOL[dt] * 10
        assert one["outcomes"] == three["outcomes"]
    finally:
        ok.orkan_free(req["h"])


def test_kept_operator_with_relabelled_qubits():
    rng = S.rng_for(5400)
    n = 7
    psi = S.haar_state_vector(rng, 1 << n)
    ops = _circuit(rng, n, 16, True)
    paulis = S.random_pauli_strings(rng, n, 4)
    a = ok.orkan_alloc(n, ok.ORKAN_C128, 3)
    b = ok.orkan_alloc(n, ok.ORKAN_C128, 3)
    try:
        for h in (a, b):
            ok.orkan_init_state(h, ok.ORKAN_INIT_PURE, psi)
        ok.orkan_relabel(a, [4, 6, 0, 2, 1, 5, 3])
        res = circuit.run_batch([{"h": a, "init": "keep", "ops": ops, "paulis": paulis}])[0]
        recs = circuit.run_circuit(b, ops)
        assert res["outcomes"] == [x for x, _ in recs]
        assert np.max(np.abs(ok.orkan_to_dense(a) - ok.orkan_to_dense(b))) <= 1e-12
        want = np.array([ok.orkan_expect_pauli(b, s) for s in paulis])
        assert np.max(np.abs(res["out"] - want)) <= 1e-12
        assert ok.orkan_get_labels(a, n) == [4, 6, 0, 2, 1, 5, 3]
    finally:
        ok.orkan_free(a)
        ok.orkan_free(b)


def test_zero_probability_and_gang_time_limit():
    n = 5
    e0 = np.zeros(1 << n, dtype=np.complex128)
    e0[0] = 1
    hs = [ok.orkan_alloc(n, ok.ORKAN_C128, 5) for _ in range(3)]
    try:
        zero = {"h": hs[0], "init": "pure", "psi0": e0, "ops": [S.op_project(0, 1), S.op_measure(0, 0.3)]}
        fine = {"h": hs[1], "init": "pure", "psi0": e0, "ops": [S.op_measure(2, 0.3)], "paulis": ["ZIIII"]}
        res = circuit.run_batch([zero, fine])
        assert res[0]["status"] == ok.ORKAN_EZEROPROB
        assert res[1]["status"] == ok.ORKAN_OK and res[1]["outcomes"] == [0] and res[1]["out"][0] == 1.0
        # a gang of two on a grid of one CTA cannot assemble: the wait runs out
        ok.orkan_batch_limits(1, 1e-3)
        try:
            res = circuit.run_batch([dict(fine, h=hs[2], gang=2)])
            assert res[0]["status"] == ok.ORKAN_ETIMEOUT
        finally:
            ok.orkan_batch_limits(0, 1.0)
        res = circuit.run_batch([dict(fine, h=hs[2], gang=2)])
        assert res[0]["status"] == ok.ORKAN_OK and res[0]["out"][0] == 1.0
    finally:
        for h in hs:
            ok.orkan_free(h)


def test_invalid_items_are_refused_before_launch():
    h = ok.orkan_alloc(4, ok.ORKAN_C128, 5)
    try:
        ok.orkan_init_observable(h, ["XZII", "IIYY"], [0.5, -1.0])
        with pytest.raises(ok.OrkanError) as e:   # a MEASURE op on the kept observable
            circuit.run_batch([{"h": h, "init": "keep", "picture": "schrodinger", "ops": [S.op_measure(1, 0.5)]}])
        assert e.value.status == ok.ORKAN_EPICTURE
        with pytest.raises(ok.OrkanError) as e:
            circuit.run_batch([{"h": h, "init": "pure", "psi0": np.ones(16) / 4,
                                "ops": [S.op_unitary(np.eye(2), [4])]}])
        assert e.value.status == ok.ORKAN_EINVAL and "batch item 0" in str(e.value)
    finally:
        ok.orkan_free(h)
