"""Checkpoint headers without a GPU: orkan_checkpoint_inspect on buffers
built here from the format documented in include/orkan.h, and its rejection
of every kind of damage (magic, version, sizes, labels, checksum, length)."""
import struct

import numpy as np
import pytest

from oracle import tiled as T
from paper_2604_15765_gb300 import orkan as ok

HDR = ok.ORKAN_CKPT_HEADER_BYTES


def _fnv_words(data: bytes) -> int:
    h = 0xcbf29ce484222325
    for (w,) in struct.iter_unpack("<Q", data):
        h = ((h ^ w) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def _checkpoint(n, dtype, m, picture, phys, data: bytes, version=1, data_bytes=None, checksum=None):
    head = b"ORKANCK1" + struct.pack("<6i", version, n, m, dtype, picture, 0)
    head += struct.pack("<64i", *(list(phys) + list(range(len(phys), 64))))
    head += struct.pack("<QQ", len(data) if data_bytes is None else data_bytes,
                        _fnv_words(data) if checksum is None else checksum)
    return head + bytes(HDR - len(head)) + data


def _data(n, m, elem):
    rng = np.random.default_rng(5)
    return rng.integers(0, 256, T.stored_bytes(n, m, elem), dtype=np.uint8).tobytes()


@pytest.mark.parametrize("n,dtype,m,elem", [(3, ok.ORKAN_C128, 5, 16), (6, ok.ORKAN_C64, 3, 8), (7, ok.ORKAN_DF64, 4, 16)])
def test_inspect_reads_a_valid_header(n, dtype, m, elem):
    phys = list(range(n))[::-1]
    buf = _checkpoint(n, dtype, m, ok.ORKAN_OBSERVABLE, phys, _data(n, m, elem))
    assert ok.orkan_checkpoint_inspect(buf) == {"n": n, "dtype": dtype, "tile_log2": m, "picture": ok.ORKAN_OBSERVABLE}


def test_inspect_rejects_damage():
    n, m = 6, 3
    data = _data(n, m, 16)
    good = _checkpoint(n, ok.ORKAN_C128, m, ok.ORKAN_STATE, range(n), data)
    flipped = bytearray(good)
    flipped[HDR + 1000] ^= 1
    bad = {
        "magic": b"ORKANCK2" + good[8:],
        "version": _checkpoint(n, ok.ORKAN_C128, m, 0, range(n), data, version=2),
        "size": _checkpoint(n, ok.ORKAN_C128, m, 0, range(n), data, data_bytes=len(data) - 16),
        "labels": _checkpoint(n, ok.ORKAN_C128, m, 0, [0, 0, 2, 3, 4, 5], data),
        "picture": _checkpoint(n, ok.ORKAN_C128, m, 7, range(n), data),
        "checksum": bytes(flipped),
        "truncated": good[:-8],
        "header_only": good[:HDR - 1],
        "dtype_size": _checkpoint(n, ok.ORKAN_C64, m, 0, range(n), data),
    }
    for what, buf in bad.items():
        with pytest.raises(ok.OrkanError) as e:
            ok.orkan_checkpoint_inspect(buf)
        assert e.value.status == ok.ORKAN_EINVAL, what
    assert ok.orkan_checkpoint_inspect(good)["n"] == n
