"""CPU oracle for the Orkan hot path (test infrastructure only).

This package is the checker, not the product.  Only the test suite, the
``smoke()`` self-check and the timed CPU baseline of ``bench.py`` may import
it; the CUDA library never calls into it and shares no code with it.

Everything here is plain NumPy / SciPy in complex128 on the full dense
``N x N`` matrix:

* :mod:`oracle.dense`  -- the Kraus map of Eq. (1) with every Kraus operator
  embedded as an explicit Kronecker product ``I (x) L (x) I`` (Sec. II-A),
  the Heisenberg adjoint, the named channels, measurement with Born
  renormalisation, Pauli expectations, traces and error measures.
* :mod:`oracle.tiled`  -- the tiled lower-triangle storage format of
  Sec. III-B (Table I sizes, tile order, element order), the bit insertion
  of Subroutine 1 and the tiled mean-value formula of Sec. III-C.
* :mod:`oracle.packed` -- the packed column-major lower-triangle format of
  Sec. III-A (the layout the tiled one is compared against).

Parity status: every function is pinned by ``tests/test_oracle_pins.py``
against closed forms, invariants, brute force or the paper's Table I.
"""
from . import dense, packed, tiled  # noqa: F401
