"""orkan_load_tiled_async: the queued upload gives the same operator as the
blocking one, later calls on the handle are ordered after it, and it may run
on a stream of its own beside another handle's passes."""
import numpy as np
import pytest

from workloads import synth as S

pytestmark = pytest.mark.gpu

ok = pytest.importorskip("paper_2604_15765_gb300.orkan")
torch = pytest.importorskip("torch")

DT = {"c128": 0, "c64": 1, "df64": 2}


@pytest.mark.parametrize("dtype", ["c128", "df64", "c64"])
def test_async_load_equals_blocking_load(dtype):
    n, m = 9, 5
    rng = S.rng_for(9400)
    U = S.haar_unitary(rng, 4)
    src = ok.orkan_alloc(n, DT[dtype], m)
    a = ok.orkan_alloc(n, DT[dtype], m)
    b = ok.orkan_alloc(n, DT[dtype], m)
    other = ok.orkan_alloc(n, DT[dtype], m)
    side = torch.cuda.Stream()
    try:
        ok.orkan_init_state(src, ok.ORKAN_INIT_DENSE, S.ginibre_state(rng, 1 << n))
        raw = np.empty(ok.orkan_bytes(n, DT[dtype], m), dtype=np.uint8)
        ok.orkan_store_tiled(src, raw)
        pinned = torch.empty(raw.size, dtype=torch.uint8, pin_memory=True)
        pinned.numpy()[:] = raw

        # reference: blocking upload, then a two-qubit gate across the tile boundary
        ok.orkan_load_tiled(a, raw, ok.ORKAN_STATE)
        ok.orkan_apply_unitary(a, [2, 7], U)
        ref = ok.orkan_to_dense(a)

        # queued upload on a stream of its own, the gate issued right behind it,
        # while another handle runs passes on the default stream
        ok.orkan_set_stream(b, side.cuda_stream)
        ok.orkan_init_state(other, ok.ORKAN_INIT_MAXMIXED)
        ok.orkan_load_tiled_async(b, pinned.numpy(), ok.ORKAN_STATE)
        for q in range(n):
            ok.orkan_depolarize(other, q, 0.1)
        ok.orkan_apply_unitary(b, [2, 7], U)
        got = ok.orkan_to_dense(b)
        assert np.array_equal(got, ref)
        assert ok.orkan_get_info(b)[3] == ok.ORKAN_STATE

        # the picture travels with the upload
        ok.orkan_load_tiled_async(b, pinned.numpy(), ok.ORKAN_OBSERVABLE)
        ok.orkan_sync(b)
        assert ok.orkan_get_info(b)[3] == ok.ORKAN_OBSERVABLE
        assert np.array_equal(ok.orkan_to_dense(b), ok.orkan_to_dense(src))

        with pytest.raises(ok.OrkanError) as e:
            ok.orkan_load_tiled_async(b, pinned.numpy(), 7)
        assert e.value.status == ok.ORKAN_EINVAL
    finally:
        for h in (src, a, b, other):
            ok.orkan_free(h)
