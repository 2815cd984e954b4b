"""The packed column-major lower-triangle format, written from its definition.

Test infrastructure only (see :mod:`oracle`).

Sec. III-A: the ``N (N + 1) / 2`` elements ``h_ij`` with ``i >= j`` are stored
column after column, each column ``j`` holding ``h_jj, h_{j+1,j}, ...,
h_{N-1,j}``.  Column ``j`` therefore starts after the ``N + (N - 1) + ... +
(N - j + 1) = j N - j (j - 1) / 2`` elements of the columns before it.  An
element above the diagonal is the conjugate of its stored partner
(``h_ij = conj(h_ji)``, Sec. II).
"""
from __future__ import annotations

import numpy as np


def packed_elements(n: int) -> int:
    N = 1 << n
    return N * (N + 1) // 2


def packed_offset(i: int, j: int, n: int):
    """(offset, conj) of h_ij: the stored partner's position and whether h_ij
    is its conjugate."""
    N = 1 << n
    conj = i < j
    p, q = (j, i) if conj else (i, j)
    return q * N - q * (q - 1) // 2 + (p - q), conj


def to_packed(H: np.ndarray) -> np.ndarray:
    """Column by column, the lower triangle of H."""
    N = H.shape[0]
    return np.concatenate([H[j:, j] for j in range(N)]).astype(np.complex128)


def from_packed(buf: np.ndarray, n: int) -> np.ndarray:
    """The hermitian matrix whose lower triangle the packed array holds."""
    N = 1 << n
    H = np.zeros((N, N), dtype=np.complex128)
    pos = 0
    for j in range(N):
        H[j:, j] = buf[pos:pos + N - j]
        pos += N - j
    low = np.tril(H, -1)
    return low + low.conj().T + np.diag(np.diag(H))
