"""orkan_alloc_external: a handle over caller-owned (torch) device memory runs
the same path as a handle that owns its buffer -- the same bits after a
circuit, within the oracle's tolerance, the operator visible in the caller's
tensor in the tiled layout -- and orkan_free leaves that memory to its owner.
"""
import numpy as np
import pytest

from oracle import dense as D
from workloads import synth as S

pytestmark = pytest.mark.gpu

ok = pytest.importorskip("paper_2604_15765_gb300.orkan")
from paper_2604_15765_gb300 import circuit  # noqa: E402

TOL = {ok.ORKAN_C128: 1e-12, ok.ORKAN_DF64: 1e-12, ok.ORKAN_C64: 1e-5}


@pytest.mark.parametrize("dtype", [ok.ORKAN_C128, ok.ORKAN_DF64, ok.ORKAN_C64])
def test_external_buffer_matches_an_owned_handle(dtype):
    import torch
    n = 7
    rng = S.rng_for(8100 + dtype)
    rho = S.ginibre_state(rng, 1 << n)
    ops = S.random_mixed_circuit(rng, n, 20, with_measure=False)
    nbytes = ok.orkan_bytes(n, dtype, 5)
    buf = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()                      # the fill is done before the handle's stream writes
    hx = ok.orkan_alloc_external(n, dtype, 5, buf.data_ptr(), nbytes)
    ho = ok.orkan_alloc(n, dtype, 5)
    try:
        for h in (hx, ho):
            ok.orkan_init_state(h, ok.ORKAN_INIT_DENSE, rho)
            circuit.run_circuit(h, ops)
            ok.orkan_sync(h)
        got, own = ok.orkan_to_dense(hx), ok.orkan_to_dense(ho)
        assert np.array_equal(got, own)
        ref, _ = D.run_circuit(rho, ops)
        assert np.max(np.abs(got - ref)) <= TOL[dtype] * 10
        raw = np.empty(nbytes, dtype=np.uint8)
        ok.orkan_store_tiled(ho, raw)
        assert np.array_equal(buf.cpu().numpy(), raw)
    finally:
        ok.orkan_free(hx)
        ok.orkan_free(ho)
    torch.cuda.synchronize()
    assert buf.cpu().numpy().any()                # still the caller's memory, still holding the operator


def test_external_buffer_too_small_is_refused():
    import torch
    n = 6
    nbytes = ok.orkan_bytes(n, ok.ORKAN_C128, 5)
    buf = torch.zeros(nbytes - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(ok.OrkanError) as e:
        ok.orkan_alloc_external(n, ok.ORKAN_C128, 5, buf.data_ptr(), nbytes - 256)
    assert e.value.status == ok.ORKAN_EINVAL
