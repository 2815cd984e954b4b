"""Continuous-batching server: every request's result is the same alone and in
the concurrent mix (bit for bit -- each kernel's grid and reduction order
depend only on the request's own operator), and matches the oracle."""
import numpy as np
import pytest

from oracle import dense as D
from workloads import synth as S

pytestmark = pytest.mark.gpu

ok = pytest.importorskip("paper_2604_15765_gb300.orkan")
from paper_2604_15765_gb300 import serving  # noqa: E402


def _requests(count=36):
    return S.serving_stream(count=count, seed=S.BASE_SEED + 40, rate=2000.0, n_range=(3, 9), depth_range=(8, 40))


@pytest.mark.parametrize("policy", ["fifo", "sjf"])
def test_results_same_alone_and_in_the_mix(policy):
    reqs = _requests()
    budget = 2 << 30
    mixed, stats = serving.serve(reqs, budget, slots=6, dtype_map={"c128": "df64"}, realtime=True, policy=policy)
    assert stats["requests"] == len(reqs)
    pool = serving.HandlePool(budget)
    try:
        for r in reqs:
            alone = serving.run_request(pool, r, {"c128": "df64"})
            assert np.array_equal(alone, mixed[r["id"]]), r["id"]
    finally:
        pool.close()
    assert stats["p99_ms"] >= stats["p50_ms"] > 0


def test_batched_results_same_alone_and_in_the_mix():
    """With the batched launch for n <= 7, a request served alone (a batch of
    one, or a slot for n > 7) gives the bits it gives in the mix."""
    reqs = _requests()
    budget = 2 << 30
    mixed, stats = serving.serve(reqs, budget, slots=4, realtime=True, batch_max_n=7)
    assert stats["requests"] == len(reqs)
    for r in reqs:
        alone, _ = serving.serve([dict(r, t=0.0)], budget, slots=1, realtime=False, batch_max_n=7)
        assert np.array_equal(alone[r["id"]], mixed[r["id"]]), r["id"]


@pytest.mark.parametrize("batch_max_n", [None, 9])
def test_served_results_match_oracle(batch_max_n):
    reqs = _requests(12)
    res, _ = serving.serve(reqs, 1 << 30, slots=4, realtime=False, batch_max_n=batch_max_n)
    for r in reqs:
        tol = 1e-10 if r["dtype"] == "c128" else 2e-4
        psi = r["psi0"]
        rho0 = np.outer(psi, psi.conj())
        if r["picture"] == "schrodinger":
            rho, _ = D.run_circuit(rho0, r["ops"], "schrodinger")
            ref = np.array([D.expect_pauli(rho, s).real for s in r["paulis"]])
        else:
            O, _ = D.run_circuit(D.pauli_sum(r["paulis"], r["coeffs"]), list(reversed(r["ops"])), "heisenberg")
            ref = np.array([D.expect(rho0, O).real])
        assert np.max(np.abs(res[r["id"]] - ref)) <= tol * max(1.0, np.abs(ref).max()), r["id"]


def test_admission_respects_memory_budget():
    reqs = [r for r in _requests(20) if r["n"] >= 6]
    one = max(ok.orkan_bytes(r["n"], 0, 5) for r in reqs) * 2
    res, stats = serving.serve(reqs, one, slots=4, realtime=False)   # only one request fits at a time
    assert stats["requests"] == len(reqs)


def test_sjf_orders_by_estimated_work():
    """Host-only ordering check: with every request present at the start and
    one slot, sjf runs them in increasing ops x 4^n."""
    reqs = _requests(10)
    done = []
    orig = serving.run_request

    def record(pool, req, *a, **k):
        done.append(req["id"])
        return orig(pool, req, *a, **k)

    serving.run_request = record
    try:
        serving.serve(reqs, 2 << 30, slots=1, realtime=False, policy="sjf")
    finally:
        serving.run_request = orig
    costs = {r["id"]: serving.request_cost(r) for r in reqs}
    assert [costs[i] for i in done] == sorted(costs[i] for i in done)
