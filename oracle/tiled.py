"""The tiled lower-triangle storage format, written from its definition.

Test infrastructure only (see :mod:`oracle`).

Sec. III-B: the ``N x N`` hermitian matrix is covered by square tiles of edge
``M = 2^m``; only tiles ``T[ti, tj]`` with ``ti >= tj`` of the
``Nt x Nt`` grid (``Nt = N / M``) are stored, tiles in row-major order in one
array, elements row-major inside a tile.  Diagonal tiles hold all ``M^2``
elements.  If ``N < M`` the matrix is padded with zeros to one ``M x M`` tile.
Total storage ``N (N + M) / 2`` elements (Table I).

The tile at grid position ``(ti, tj)`` therefore starts at element
``(ti (ti + 1) / 2 + tj) * M^2`` (the tile offsets used in Algorithm 3).

Subroutine 1 (insertBits) is restated here by its meaning -- build the
global index bit by bit, taking the next bit of ``a`` at every position in
``A`` and the next bit of ``s`` elsewhere -- so that the library's shift-based
implementation can be checked against it.
"""
from __future__ import annotations

import numpy as np


def tile_edge(m: int) -> int:
    return 1 << m


def num_tile_rows(n: int, m: int) -> int:
    """Nt = N / M, or 1 when N < M (zero padding to a single tile)."""
    return max(1, (1 << n) >> m)


def num_tiles(n: int, m: int) -> int:
    nt = num_tile_rows(n, m)
    return nt * (nt + 1) // 2


def stored_elements(n: int, m: int) -> int:
    """N (N + M) / 2, or M^2 when N < M (Table I)."""
    return num_tiles(n, m) * (1 << m) ** 2


def stored_bytes(n: int, m: int, elem_bytes: int = 16) -> int:
    return stored_elements(n, m) * elem_bytes


def tile_start(ti: int, tj: int, m: int) -> int:
    """Element offset of tile (ti, tj), ti >= tj, in the contiguous array."""
    assert ti >= tj
    return (ti * (ti + 1) // 2 + tj) * (1 << m) ** 2


def to_tiled(H: np.ndarray, m: int) -> np.ndarray:
    """Store the lower triangle of H at tile granularity (Sec. III-B)."""
    N = H.shape[0]
    M = 1 << m
    n = int(np.log2(N))
    if N < M:
        P = np.zeros((M, M), dtype=H.dtype)
        P[:N, :N] = H
        H = P
    nt = num_tile_rows(n, m)
    out = np.zeros(stored_elements(n, m), dtype=H.dtype)
    for ti in range(nt):
        for tj in range(ti + 1):
            s = tile_start(ti, tj, m)
            out[s:s + M * M] = H[ti * M:(ti + 1) * M, tj * M:(tj + 1) * M].reshape(-1)
    return out


def from_tiled(buf: np.ndarray, n: int, m: int) -> np.ndarray:
    """Rebuild the dense N x N matrix.  Element (i, j) with i >= j is read from
    its stored tile; element (i, j) with i < j is the conjugate of (j, i),
    also inside diagonal tiles (the lower triangle is authoritative)."""
    N = 1 << n
    M = 1 << m
    nt = num_tile_rows(n, m)
    full = np.zeros((nt * M, nt * M), dtype=buf.dtype)
    for ti in range(nt):
        for tj in range(ti + 1):
            s = tile_start(ti, tj, m)
            full[ti * M:(ti + 1) * M, tj * M:(tj + 1) * M] = buf[s:s + M * M].reshape(M, M)
    full = full[:N, :N]
    lower = np.tril(full)
    return lower + np.tril(full, -1).conj().T


def element_offset(i: int, j: int, n: int, m: int):
    """(offset, conjugate?) of element (i, j) in the tiled array."""
    conj = False
    if i < j:
        i, j, conj = j, i, True
    M = 1 << m
    off = tile_start(i >> m, j >> m, m) + (i & (M - 1)) * M + (j & (M - 1))
    return off, conj


def insert_bits(s: int, a: int, A) -> int:
    """Subroutine 1 by its meaning: bits of ``a`` go, in order, to the sorted
    positions ``A``; the bits of ``s`` fill the other positions in order."""
    A = sorted(int(p) for p in A)
    width = max(A) + 1 if A else 0
    out = 0
    ia = 0
    is_ = 0
    pos = 0
    # positions below and between the active ones, then all of s's higher bits
    while pos < width or (s >> is_):
        if ia < len(A) and pos == A[ia]:
            out |= ((a >> ia) & 1) << pos
            ia += 1
        else:
            out |= ((s >> is_) & 1) << pos
            is_ += 1
        pos += 1
    return out


def tiled_mean_value(rho_buf, O_buf, n: int, m: int) -> float:
    """Sec. III-C: tr(rho O) from the tiles as Frobenius products, the diagonal
    tiles once and the strictly-lower tiles (ti > tj) twice.  (The printed
    second sum runs over ti >= tj, which would count the diagonal tiles three
    times; the strict reading is the one that equals the trace.)"""
    M = 1 << m
    nt = num_tile_rows(n, m)
    total = 0.0
    for ti in range(nt):
        for tj in range(ti + 1):
            s = tile_start(ti, tj, m)
            f = np.vdot(O_buf[s:s + M * M], rho_buf[s:s + M * M]).real
            total += f if ti == tj else 2.0 * f
    return float(total)
