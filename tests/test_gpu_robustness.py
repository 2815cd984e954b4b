"""Failure handling and checkpoints on the GPU, without faulting it.

* An allocation far beyond the device (n = 24 complex128: 2.25 PB of tiles)
  fails on the host side of cudaMalloc with ORKAN_ENOMEM and a message, and
  the process and the library stay usable.
* Checkpoints (header + raw tiled array) round-trip an operator with its
  picture and qubit labels, and a checkpoint is refused by a handle of
  another n, tile size or dtype, or when damaged, leaving the handle as it
  was.
"""
import numpy as np
import pytest

from workloads import synth as S

pytestmark = pytest.mark.gpu

ok = pytest.importorskip("paper_2604_15765_gb300.orkan")
from paper_2604_15765_gb300 import circuit  # noqa: E402


def test_oversized_alloc_is_enomem_and_the_library_stays_usable():
    with pytest.raises(ok.OrkanError) as e:
        ok.orkan_alloc(24, ok.ORKAN_C128, 5)
    assert e.value.status == ok.ORKAN_ENOMEM
    assert "cudaMalloc" in str(e.value)
    h = ok.orkan_alloc(6, ok.ORKAN_C128, 5)
    try:
        ok.orkan_init_state(h, ok.ORKAN_INIT_MAXMIXED)
        ok.orkan_apply_unitary(h, [0, 5], S.haar_unitary(S.rng_for(1), 4))
        assert ok.orkan_trace(h) == pytest.approx(1.0, abs=1e-14)
    finally:
        ok.orkan_free(h)


@pytest.mark.parametrize("dtype,m", [(ok.ORKAN_C128, 5), (ok.ORKAN_DF64, 3), (ok.ORKAN_C64, 4)])
def test_checkpoint_round_trip_keeps_labels_and_picture(dtype, m):
    n = 7
    rng = S.rng_for(880 + dtype)
    strings, coeffs = S.random_pauli_sum(rng, n, 16)
    a = ok.orkan_alloc(n, dtype, m)
    b = ok.orkan_alloc(n, dtype, m)
    try:
        ok.orkan_init_observable(a, strings, coeffs)
        circuit.run_circuit(a, S.random_mixed_circuit(rng, n, 20, with_measure=False), "heisenberg")
        ok.orkan_relabel(a, [3, 0, 6, 1, 5, 2, 4])
        want = ok.orkan_to_dense(a)
        labels = ok.orkan_get_labels(a, n)
        buf = ok.orkan_checkpoint_save(a)
        assert buf.size == ok.ORKAN_CKPT_HEADER_BYTES + ok.orkan_bytes(n, dtype, m)
        assert ok.orkan_checkpoint_inspect(buf) == {"n": n, "dtype": dtype, "tile_log2": m,
                                                    "picture": ok.ORKAN_OBSERVABLE}
        ok.orkan_init_state(b, ok.ORKAN_INIT_ZERO)
        ok.orkan_checkpoint_load(b, buf)
        assert ok.orkan_get_labels(b, n) == labels
        assert ok.orkan_get_info(b)[3] == ok.ORKAN_OBSERVABLE
        assert np.array_equal(ok.orkan_to_dense(b), want)
        # the restored handle keeps evolving like the original
        U = S.haar_unitary(rng, 4)
        for h in (a, b):
            ok.orkan_apply_unitary(h, [2, 5], U)
        assert np.array_equal(ok.orkan_to_dense(a), ok.orkan_to_dense(b))
    finally:
        ok.orkan_free(a)
        ok.orkan_free(b)


def test_checkpoint_refused_by_a_mismatched_handle_or_when_damaged():
    n = 6
    rng = S.rng_for(890)
    a = ok.orkan_alloc(n, ok.ORKAN_C128, 5)
    others = [ok.orkan_alloc(n + 1, ok.ORKAN_C128, 5), ok.orkan_alloc(n, ok.ORKAN_DF64, 5),
              ok.orkan_alloc(n, ok.ORKAN_C128, 4)]
    try:
        ok.orkan_init_state(a, ok.ORKAN_INIT_PURE, S.haar_state_vector(rng, 1 << n))
        buf = ok.orkan_checkpoint_save(a)
        for h in others:
            ok.orkan_init_state(h, ok.ORKAN_INIT_MAXMIXED)
            before = ok.orkan_to_dense(h)
            with pytest.raises(ok.OrkanError) as e:
                ok.orkan_checkpoint_load(h, buf)
            assert e.value.status == ok.ORKAN_EINVAL
            assert "the handle has" in str(e.value)
            assert np.array_equal(ok.orkan_to_dense(h), before)
        ok.orkan_apply_unitary(a, [1], S.haar_unitary(rng, 2))
        before = ok.orkan_to_dense(a)
        damaged = buf.copy()
        damaged[ok.ORKAN_CKPT_HEADER_BYTES + 17] ^= 0x40
        with pytest.raises(ok.OrkanError) as e:
            ok.orkan_checkpoint_load(a, damaged)
        assert e.value.status == ok.ORKAN_EINVAL and "checksum" in str(e.value)
        with pytest.raises(ok.OrkanError):
            ok.orkan_checkpoint_load(a, buf[:-16])
        assert np.array_equal(ok.orkan_to_dense(a), before)
    finally:
        ok.orkan_free(a)
        for h in others:
            ok.orkan_free(h)
