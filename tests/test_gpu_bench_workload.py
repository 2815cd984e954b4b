"""The timed configuration of bench.py against the oracle: the per-op sweep of
both pictures (fusion 8, composition and the fold on), the Z measurement, the
Pauli readouts, the trace and tr(rho O), issued exactly as bench.Runner issues
them, from the same workload builder as the n = 14 headline, at n = 9 where
the dense oracle is quick -- two steps, every dtype, readouts and both final
operators."""
import importlib.util
import os

import numpy as np
import pytest

from oracle import dense as D

pytestmark = pytest.mark.gpu

ok = pytest.importorskip("paper_2604_15765_gb300.orkan")
from paper_2604_15765_gb300 import circuit  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL = {"c128": 1e-12, "df64": 1e-12, "c64": 1e-5}


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
def test_bench_steps_match_the_oracle(dtype):
    import torch
    bench = _bench()
    n = 9
    wl = bench.make_workload(n)
    r = bench.Runner(ok, circuit, wl, n, 5, dtype, 8, True, torch.cuda.current_stream().cuda_stream)
    try:
        rho = np.outer(wl["psi"], wl["psi"].conj())
        for q in range(n):
            rho = D.depolarize(rho, q, 0.1)
        O = D.pauli_sum(*wl["obs"])
        for step in range(2):
            got = np.array(r.step())
            rho, _ = D.run_circuit(rho, wl["ops"], "schrodinger")
            rho, _, pb = D.measure(rho, step % n, float(wl["us"][step % len(wl["us"])]))
            O, _ = D.run_circuit(O, list(reversed(wl["ops"])), "heisenberg")
            want = np.array([pb] + [D.expect_pauli(rho, s).real for s in wl["paulis"]] + [D.trace(rho).real]
                            + [D.expect(rho, O).real])
            scale = max(1.0, float(np.max(np.abs(O))))
            assert np.max(np.abs(got - want)) <= TOL[dtype] * scale * 100, (step, got, want)
        assert np.max(np.abs(ok.orkan_to_dense(r.rho) - rho)) <= TOL[dtype] * 10
        assert np.max(np.abs(ok.orkan_to_dense(r.O) - O)) <= TOL[dtype] * scale * 10
    finally:
        r.free()
