"""The allocation-free Pauli readout, orkan_expect_paulis_noalloc.

It serves callers that must not allocate device memory themselves (a host
framework that owns all device memory through its own pool, a serving loop
that cannot afford an allocation's possible device synchronisation, a plugin
that only receives the tiled operator's device pointer).  Its scratch is one
fixed device array shared by every call, so this test calls it twice in a row
-- and once more with a shorter batch -- and checks each result against the
existing entry point orkan_expect_pauli bit for bit (the two use the same
grid and reduction order), and once against the oracle within the parity
tolerance of the other GPU tests.  A relabelled handle checks that the
strings act on physical bit positions.  The file is named to be collected
last.
"""
import numpy as np
import pytest

from workloads import synth as S

pytestmark = pytest.mark.gpu

ok = pytest.importorskip("paper_2604_15765_gb300.orkan")
from paper_2604_15765_gb300 import circuit  # noqa: E402
from oracle import dense as D  # noqa: E402

TOL = {ok.ORKAN_C128: 1e-12, ok.ORKAN_DF64: 1e-12, ok.ORKAN_C64: 1e-5}


def _physical(s, phys):
    """Move character q of a logical string to position phys[q]."""
    out = ["I"] * len(s)
    for q, ch in enumerate(s):
        out[phys[q]] = ch
    return "".join(out)


@pytest.mark.parametrize("dtype,n,m", [(ok.ORKAN_C128, 10, 5), (ok.ORKAN_DF64, 12, 5), (ok.ORKAN_C64, 9, 3),
                                       (ok.ORKAN_C128, 3, 5)])
def test_noalloc_pauli_readout_matches_existing_entry_point(dtype, n, m):
    rng = S.rng_for(7000 + n)
    h = ok.orkan_alloc(n, dtype, m)
    try:
        psi = S.haar_state_vector(rng, 1 << n)
        ops = S.random_mixed_circuit(rng, n, 30, with_measure=False)
        ok.orkan_init_state(h, ok.ORKAN_INIT_PURE, psi)
        circuit.run_circuit(h, ops)
        ok.orkan_sync(h)
        strings = S.random_pauli_strings(rng, n, 40) + ["I" * n, "Y" * n, "Z" * n, "X" * n]
        ref = np.array([ok.orkan_expect_pauli(h, s) for s in strings])
        ptr = ok.orkan_device_ptr(h)
        for _ in range(2):   # two calls in a row share the scratch array
            got = ok.orkan_expect_paulis_noalloc(ptr, n, dtype, m, strings)
            assert np.array_equal(got, ref)
        got = ok.orkan_expect_paulis_noalloc(ptr, n, dtype, m, strings[:5])
        assert np.array_equal(got, ref[:5])
        if n <= 10:   # once against the oracle
            rho = D.run_circuit(np.outer(psi, psi.conj()), ops)[0]
            want = np.array([D.expect_pauli(rho, s).real for s in strings])
            assert np.max(np.abs(got[:5] - want[:5])) <= TOL[dtype] * 10
        with pytest.raises(ok.OrkanError) as e:
            ok.orkan_expect_paulis_noalloc(ptr, n, dtype, m, strings * 2)   # 88 > 64 strings
        assert e.value.status == ok.ORKAN_EINVAL
        assert "ORKAN_NOALLOC_MAX_STRINGS" in str(e.value)
    finally:
        ok.orkan_free(h)


@pytest.mark.parametrize("dtype", [ok.ORKAN_C128, ok.ORKAN_C64])
def test_noalloc_pauli_readout_on_relabelled_handle(dtype):
    """After orkan_relabel the device array is indexed by physical positions:
    a logical string moved through orkan_get_labels gives orkan_expect_pauli's
    value for the logical string, bit for bit."""
    n, m = 8, 3
    rng = S.rng_for(7100 + dtype)
    h = ok.orkan_alloc(n, dtype, m)
    try:
        ok.orkan_init_state(h, ok.ORKAN_INIT_PURE, S.haar_state_vector(rng, 1 << n))
        circuit.run_circuit(h, S.random_mixed_circuit(rng, n, 20, with_measure=False))
        ok.orkan_relabel(h, [5, 7, 0, 6, 1, 2, 4, 3])
        ok.orkan_sync(h)
        phys = ok.orkan_get_labels(h, n)
        assert phys != list(range(n))
        strings = S.random_pauli_strings(rng, n, 24)
        ref = np.array([ok.orkan_expect_pauli(h, s) for s in strings])
        got = ok.orkan_expect_paulis_noalloc(ok.orkan_device_ptr(h), n, dtype, m,
                                             [_physical(s, phys) for s in strings])
        assert np.array_equal(got, ref)
    finally:
        ok.orkan_free(h)
