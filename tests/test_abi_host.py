"""The C-ABI library without a GPU: it loads, exports every entry point that
include/orkan.h declares, and its host-only functions (layout, bit insertion,
Pauli transfer matrices) agree with the oracle."""
import itertools
import os
import re

import numpy as np
import pytest

from oracle import dense as D
from oracle import tiled as T
from paper_2604_15765_gb300 import orkan as ok
from workloads import synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "orkan.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(orkan_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 30
    for name in names:
        assert hasattr(ok._lib, name), name
        assert name in ok.EXPORTED, f"binding lacks {name}"


def test_bytes_follow_table1_formula():
    for n in range(1, 20):
        assert ok.orkan_bytes(n, ok.ORKAN_C128, 2) == 0           # tiles below M = 8 are not supported
        for m in (3, 4, 5):
            assert ok.orkan_bytes(n, ok.ORKAN_C128, m) == T.stored_bytes(n, m, 16)
            assert ok.orkan_bytes(n, ok.ORKAN_DF64, m) == T.stored_bytes(n, m, 16)
            assert ok.orkan_bytes(n, ok.ORKAN_C64, m) == T.stored_bytes(n, m, 8)
            assert ok.orkan_num_tiles(n, m) == T.num_tiles(n, m)
    assert ok.orkan_bytes(5, ok.ORKAN_C128, 0) == 16384          # default m = 5
    assert ok.orkan_bytes(0, ok.ORKAN_C128, 5) == 0               # invalid n
    assert ok.orkan_bytes(4, 7, 5) == 0                           # invalid dtype
    assert ok.orkan_bytes(4, ok.ORKAN_C128, 6) == 0               # tile too large (m <= 5)


@pytest.mark.parametrize("n,m", [(1, 5), (3, 3), (5, 5), (6, 3), (7, 4), (8, 5)])
def test_element_offset_matches_oracle(n, m):
    for i in range(1 << n):
        for j in range(1 << n):
            assert ok.orkan_element_offset(n, m, i, j) == T.element_offset(i, j, n, m)
    assert ok.orkan_element_offset(n, m, 1 << n, 0)[0] == -1


def test_insert_bits_matches_oracle():
    for n in range(1, 7):
        for k in range(1, min(3, n) + 1):
            for A in itertools.combinations(range(n), k):
                for s in range(1 << (n - k)):
                    for a in range(1 << k):
                        assert ok.orkan_insert_bits(s, a, A) == T.insert_bits(s, a, A)


def _pauli(a, k):
    P = np.ones((1, 1), dtype=np.complex128)
    for l in reversed(range(k)):
        P = np.kron(P, [D.I2, D.X, D.Y, D.Z][(a >> (2 * l)) & 3])
    return P


@pytest.mark.parametrize("k,r", [(1, 1), (1, 2), (1, 4), (2, 1), (2, 3)])
def test_ptm_reproduces_the_kraus_map(k, r):
    rng = S.rng_for(500 + 10 * k + r)
    d = 1 << k
    kraus = [rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d)) for _ in range(r)]
    B = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    for adjoint in (False, True):
        R = ok.orkan_ptm(k, kraus, adjoint)
        expect = D.apply_kraus(B, kraus, list(range(k)), "heisenberg" if adjoint else "schrodinger")
        z = np.array([np.trace(_pauli(b, k) @ B) / d for b in range(4 ** k)])
        got = sum((R[a] @ z) * _pauli(a, k) for a in range(4 ** k))
        assert np.max(np.abs(got - expect)) < 1e-12


def test_alloc_without_gpu_reports_no_device():
    from conftest import gpu_available
    if gpu_available():
        pytest.skip("a GPU is present")
    with pytest.raises(ok.OrkanError) as e:
        ok.orkan_alloc(4, ok.ORKAN_C128, 5)
    assert e.value.status == ok.ORKAN_ENODEV


def test_external_buffer_must_be_256_byte_aligned():
    """orkan_alloc_external refuses a null or unaligned device pointer before
    touching the device (the kernels move 16-byte granules and 8 KiB tiles)."""
    for ptr in (0, 0x10008, 0x10010, 0x10080):
        with pytest.raises(ok.OrkanError) as e:
            ok.orkan_alloc_external(4, ok.ORKAN_C128, 5, ptr, 1 << 20)
        assert e.value.status == ok.ORKAN_EINVAL


def test_serving_pool_refuses_a_request_larger_than_its_budget():
    """A request whose operators can never fit the memory budget fails at
    admission (host-side, before any device call) instead of waiting forever."""
    from paper_2604_15765_gb300 import serving
    pool = serving.HandlePool(budget_bytes=ok.orkan_bytes(10, ok.ORKAN_C128, 5) + 1)
    with pytest.raises(ValueError):
        pool.acquire(11, "c128", 1)
    with pytest.raises(ValueError):
        pool.acquire(10, "c128", 2)          # a Heisenberg request holds two operators


def test_packed_layout_matches_oracle():
    from oracle import packed as PK
    for n in range(1, 12):
        assert ok.orkan_packed_bytes(n, ok.ORKAN_C128) == PK.packed_elements(n) * 16
        assert ok.orkan_packed_bytes(n, ok.ORKAN_DF64) == PK.packed_elements(n) * 16
        assert ok.orkan_packed_bytes(n, ok.ORKAN_C64) == PK.packed_elements(n) * 8
    assert ok.orkan_packed_bytes(0, ok.ORKAN_C128) == 0
    assert ok.orkan_packed_bytes(3, 9) == 0
    for n in (1, 3, 5):
        for i in range(1 << n):
            for j in range(1 << n):
                assert ok.orkan_packed_offset(n, i, j) == PK.packed_offset(i, j, n)
    assert ok.orkan_packed_offset(3, 8, 0)[0] == -1


def test_packed_calls_validate_before_any_launch():
    """Argument errors are reported without touching a device."""
    U = np.eye(2, dtype=np.complex128)
    with pytest.raises(ok.OrkanError):
        ok.orkan_packed_apply_unitary(0, 3, ok.ORKAN_C128, [0], U)            # null array
    with pytest.raises(ok.OrkanError):
        ok.orkan_packed_apply_unitary(64, 3, ok.ORKAN_C128, [3], U)           # qubit out of range
    with pytest.raises(ok.OrkanError):
        ok.orkan_packed_apply_unitary(64, 3, ok.ORKAN_C128, [0, 1, 2], np.eye(8))   # k = 3
    with pytest.raises(ok.OrkanError):
        ok.orkan_packed_apply_kraus(64, 3, ok.ORKAN_C128, [0, 1], np.stack([np.eye(4) * 0.5] * 2))  # r > 1, k = 2
    with pytest.raises(ok.OrkanError):
        ok.orkan_packed_depolarize(64, 3, ok.ORKAN_C128, 0, 1.5)


def test_batch_and_tensor_entry_points_validate_on_the_host():
    """orkan_batch_limits checks its arguments without a GPU; an empty batch
    is a no-op; a NULL handle is refused by orkan_set_tensor."""
    import ctypes as C
    with pytest.raises(ok.OrkanError) as e:
        ok.orkan_batch_limits(-1, 1.0)
    assert e.value.status == ok.ORKAN_EINVAL
    with pytest.raises(ok.OrkanError):
        ok.orkan_batch_limits(0, 0.0)
    with pytest.raises(ok.OrkanError):
        ok.orkan_batch_limits(0, 100.0)
    ok.orkan_batch_limits(4, 0.5)
    ok.orkan_batch_limits(0, 1.0)
    assert ok._lib.orkan_run_batch(0, None, None) == ok.ORKAN_OK
    assert ok._lib.orkan_run_batch(-1, None, None) == ok.ORKAN_EINVAL
    assert ok._lib.orkan_set_tensor(C.c_void_p(0), 1) == ok.ORKAN_EINVAL
