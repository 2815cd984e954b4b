"""The allocation-free Pauli readout, orkan_expect_paulis_noalloc.

It serves callers that must not allocate device memory themselves (a host
framework that owns all device memory through its own pool, a serving loop
that cannot afford an allocation's possible device synchronisation, a plugin
that only receives the tiled operator's device pointer).  Its scratch is one
fixed device array shared by every call, so this test calls it twice in a row
-- and once more with a shorter batch -- and checks each result against the
existing entry point orkan_expect_pauli within the parity tolerance of the
other GPU tests.  The file is named to be collected last.
"""
import numpy as np
import pytest

from workloads import synth as S

pytestmark = pytest.mark.gpu

ok = pytest.importorskip("paper_2604_15765_gb300.orkan")
from paper_2604_15765_gb300 import circuit  # noqa: E402

TOL = {ok.ORKAN_C128: 1e-12, ok.ORKAN_DF64: 1e-12, ok.ORKAN_C64: 1e-5}


@pytest.mark.parametrize("dtype,n,m", [(ok.ORKAN_C128, 10, 5), (ok.ORKAN_DF64, 12, 5), (ok.ORKAN_C64, 9, 3),
                                       (ok.ORKAN_C128, 3, 5)])
def test_noalloc_pauli_readout_matches_existing_entry_point(dtype, n, m):
    rng = S.rng_for(7000 + n)
    h = ok.orkan_alloc(n, dtype, m)
    try:
        ok.orkan_init_state(h, ok.ORKAN_INIT_PURE, S.haar_state_vector(rng, 1 << n))
        circuit.run_circuit(h, S.random_mixed_circuit(rng, n, 30, with_measure=False))
        ok.orkan_sync(h)
        strings = S.random_pauli_strings(rng, n, 40) + ["I" * n, "Y" * n, "Z" * n, "X" * n]
        ref = np.array([ok.orkan_expect_pauli(h, s) for s in strings])
        ptr = ok.orkan_device_ptr(h)
        tol = TOL[dtype] * 10 * max(1.0, float(np.max(np.abs(ref))))
        for _ in range(2):   # two calls in a row share the scratch array
            got = ok.orkan_expect_paulis_noalloc(ptr, n, dtype, m, strings)
            assert np.max(np.abs(got - ref)) <= tol
        got = ok.orkan_expect_paulis_noalloc(ptr, n, dtype, m, strings[:5])
        assert np.max(np.abs(got - ref[:5])) <= tol
        with pytest.raises(ok.OrkanError) as e:
            ok.orkan_expect_paulis_noalloc(ptr, n, dtype, m, strings * 2)   # 88 > 64 strings
        assert e.value.status == ok.ORKAN_EINVAL
        assert "ORKAN_NOALLOC_MAX_STRINGS" in str(e.value)
    finally:
        ok.orkan_free(h)
