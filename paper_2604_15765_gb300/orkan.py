"""ctypes binding of the Orkan C ABI (include/orkan.h), same names, marshalling only.

Every function here converts Python / NumPy arguments to the C types, calls
the entry point of ``liborkan_gb300.so`` with the same name, and raises
:class:`OrkanError` on a non-zero status.  No computation happens in Python:
if the shared library is missing the import fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liborkan_gb300.so")

ORKAN_C128, ORKAN_C64, ORKAN_DF64 = 0, 1, 2
ORKAN_STATE, ORKAN_OBSERVABLE = 0, 1
ORKAN_INIT_ZERO, ORKAN_INIT_MAXMIXED, ORKAN_INIT_DENSE, ORKAN_INIT_PURE = 0, 1, 2, 3
ORKAN_OK, ORKAN_EINVAL, ORKAN_ENOMEM, ORKAN_ECUDA, ORKAN_EZEROPROB, ORKAN_EPICTURE, ORKAN_ENODEV = 0, -1, -2, -3, -4, -5, -6
ORKAN_ETIMEOUT = -7
DTYPES = {"c128": ORKAN_C128, "c64": ORKAN_C64, "df64": ORKAN_DF64}


class OrkanError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run paper_2604_15765_gb300.build.build() "
                      "(there is no CPU fallback for the Orkan path)")
_lib = C.CDLL(LIB_PATH)

_h = C.c_void_p


class OrkanOp(C.Structure):
    """orkan_op of include/orkan.h."""
    _fields_ = [("kind", C.c_int), ("k", C.c_int), ("qubits", C.c_int * 3), ("r", C.c_int), ("outcome", C.c_int),
                ("param", C.c_double), ("mats", C.POINTER(C.c_double))]


class OrkanBatchItem(C.Structure):
    """orkan_batch_item of include/orkan.h."""
    _fields_ = [("h", C.c_void_p), ("init", C.c_int), ("init_data", C.POINTER(C.c_double)), ("nterms", C.c_int),
                ("terms", C.c_char_p), ("coeffs", C.POINTER(C.c_double)), ("nops", C.c_int),
                ("ops", C.POINTER(OrkanOp)), ("npaulis", C.c_int), ("paulis", C.c_char_p),
                ("psi", C.POINTER(C.c_double)), ("out", C.POINTER(C.c_double)), ("outcomes", C.POINTER(C.c_int)),
                ("probs", C.POINTER(C.c_double)), ("gang", C.c_int), ("status", C.c_int)]


ORKAN_BATCH_KEEP, ORKAN_BATCH_PAULI_SUM = -1, 4
ORKAN_OP_UNITARY, ORKAN_OP_KRAUS, ORKAN_OP_DEPOLARIZE, ORKAN_OP_DEPHASE = 0, 1, 2, 3
ORKAN_OP_AMPDAMP, ORKAN_OP_MEASURE, ORKAN_OP_PROJECT = 4, 5, 6
_i64 = C.c_int64
_pd = C.POINTER(C.c_double)
_pi = C.POINTER(C.c_int)

_SIGS = {
    "orkan_strerror": (C.c_char_p, [C.c_int]),
    "orkan_last_error": (C.c_char_p, []),
    "orkan_bytes": (C.c_size_t, [C.c_int, C.c_int, C.c_int]),
    "orkan_num_tiles": (_i64, [C.c_int, C.c_int]),
    "orkan_element_offset": (_i64, [C.c_int, C.c_int, _i64, _i64, _pi]),
    "orkan_insert_bits": (C.c_uint64, [C.c_uint64, C.c_uint64, C.c_int, _pi]),
    "orkan_ptm": (C.c_int, [C.c_int, C.c_int, _pd, C.c_int, _pd]),
    "orkan_alloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(_h)]),
    "orkan_alloc_external": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_size_t, C.POINTER(_h)]),
    "orkan_free": (C.c_int, [_h]),
    "orkan_set_stream": (C.c_int, [_h, C.c_void_p]),
    "orkan_set_fusion": (C.c_int, [_h, C.c_int, C.c_int]),
    "orkan_set_tensor": (C.c_int, [_h, C.c_int]),
    "orkan_get_info": (C.c_int, [_h, _pi, _pi, _pi, _pi]),
    "orkan_autotune": (C.c_int, [C.c_int, C.c_int, _pi, _pi]),
    "orkan_device_ptr": (C.c_void_p, [_h]),
    "orkan_init_state": (C.c_int, [_h, C.c_int, _pd]),
    "orkan_init_observable": (C.c_int, [_h, C.c_int, C.c_char_p, _pd]),
    "orkan_set_picture": (C.c_int, [_h, C.c_int]),
    "orkan_load_tiled": (C.c_int, [_h, C.c_void_p, C.c_int]),
    "orkan_store_tiled": (C.c_int, [_h, C.c_void_p]),
    "orkan_load_tiled_async": (C.c_int, [_h, C.c_void_p, C.c_int]),
    "orkan_apply_unitary": (C.c_int, [_h, C.c_int, _pi, _pd]),
    "orkan_apply_kraus": (C.c_int, [_h, C.c_int, _pi, C.c_int, _pd]),
    "orkan_depolarize": (C.c_int, [_h, C.c_int, C.c_double]),
    "orkan_dephase": (C.c_int, [_h, C.c_int, C.c_double]),
    "orkan_amplitude_damp": (C.c_int, [_h, C.c_int, C.c_double]),
    "orkan_measure": (C.c_int, [_h, C.c_int, C.c_double, _pi, _pd]),
    "orkan_project": (C.c_int, [_h, C.c_int, C.c_int]),
    "orkan_run_circuit": (C.c_int, [_h, C.c_int, C.POINTER(OrkanOp), _pi, _pd, _pi]),
    "orkan_trace": (C.c_int, [_h, _pd, _pd]),
    "orkan_expect_pauli": (C.c_int, [_h, C.c_char_p, _pd]),
    "orkan_expect": (C.c_int, [_h, _h, _pd]),
    "orkan_to_dense": (C.c_int, [_h, _pd]),
    "orkan_get_elements": (C.c_int, [_h, _i64, C.POINTER(_i64), C.POINTER(_i64), _pd]),
    "orkan_flush": (C.c_int, [_h]),
    "orkan_sync": (C.c_int, [_h]),
    "orkan_stats": (C.c_int, [_h, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i64)]),
    "orkan_capture_begin": (C.c_int, [_h]),
    "orkan_capture_end": (C.c_int, [_h, C.POINTER(C.c_void_p)]),
    "orkan_graph_launch": (C.c_int, [_h, C.c_void_p]),
    "orkan_graph_free": (C.c_int, [C.c_void_p]),
    "orkan_set_timing": (C.c_int, [_h, C.c_int]),
    "orkan_pass_time": (C.c_int, [_h, _pd, C.POINTER(_i64)]),
    "orkan_pass_work": (C.c_int, [_h, _pd, _pd]),
    "orkan_expect_paulis_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_char_p, _pd,
                                              C.c_void_p]),
    "orkan_probe_pipes": (C.c_int, [_pd, C.c_void_p, C.c_size_t]),
    "orkan_relabel": (C.c_int, [_h, _pi]),
    "orkan_get_labels": (C.c_int, [_h, _pi]),
    "orkan_set_relabel": (C.c_int, [_h, C.c_int]),
    "orkan_packed_bytes": (C.c_size_t, [C.c_int, C.c_int]),
    "orkan_packed_offset": (_i64, [C.c_int, _i64, _i64, _pi]),
    "orkan_packed_apply_unitary": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, _pi, _pd, C.c_void_p]),
    "orkan_packed_apply_kraus": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, _pi, C.c_int, _pd,
                                           C.c_void_p]),
    "orkan_packed_depolarize": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_void_p]),
    "orkan_packed_from_tiled": (C.c_int, [_h, C.c_void_p]),
    "orkan_packed_to_tiled": (C.c_int, [_h, C.c_void_p]),
    "orkan_run_batch": (C.c_int, [C.c_int, C.POINTER(OrkanBatchItem), C.c_void_p]),
    "orkan_batch_limits": (C.c_int, [C.c_int, C.c_double]),
    "orkan_checkpoint_bytes": (C.c_size_t, [_h]),
    "orkan_checkpoint_save": (C.c_int, [_h, C.c_void_p, C.c_size_t]),
    "orkan_checkpoint_load": (C.c_int, [_h, C.c_void_p, C.c_size_t]),
    "orkan_checkpoint_inspect": (C.c_int, [C.c_void_p, C.c_size_t, _pi, _pi, _pi, _pi]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


def _check(status: int, where: str):
    if status != ORKAN_OK:
        msg = _lib.orkan_last_error().decode() or _lib.orkan_strerror(status).decode()
        raise OrkanError(status, where, msg)


def _cplx(a, d=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    if d is not None:
        a = a.reshape(-1, d, d)
    return a


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_pd)


def _qubits(qubits):
    arr = (C.c_int * len(qubits))(*[int(q) for q in qubits])
    return arr


# ------------------------------------------------------------------ layout
def orkan_bytes(n: int, dtype: int = ORKAN_C128, tile_log2: int = 5) -> int:
    return int(_lib.orkan_bytes(n, dtype, tile_log2))


def orkan_num_tiles(n: int, tile_log2: int = 5) -> int:
    return int(_lib.orkan_num_tiles(n, tile_log2))


def orkan_element_offset(n: int, tile_log2: int, i: int, j: int):
    cj = C.c_int(0)
    off = _lib.orkan_element_offset(n, tile_log2, i, j, C.byref(cj))
    return int(off), bool(cj.value)


def orkan_insert_bits(s: int, a: int, pos) -> int:
    return int(_lib.orkan_insert_bits(s, a, len(pos), _qubits(pos)))


def orkan_ptm(k: int, kraus, adjoint: bool = False) -> np.ndarray:
    K = _cplx(kraus, 1 << k)
    out = np.zeros((4 ** k, 4 ** k))
    _check(_lib.orkan_ptm(k, K.shape[0], _dptr(K.view(np.float64)), int(adjoint), _dptr(out)), "orkan_ptm")
    return out


# ------------------------------------------------------------------ lifetime
def orkan_alloc(n: int, dtype: int = ORKAN_C128, tile_log2: int = 5):
    h = _h()
    _check(_lib.orkan_alloc(n, dtype, tile_log2, C.byref(h)), "orkan_alloc")
    return h


def orkan_alloc_external(n: int, dtype: int, tile_log2: int, dev_ptr: int, nbytes: int):
    h = _h()
    _check(_lib.orkan_alloc_external(n, dtype, tile_log2, C.c_void_p(dev_ptr), nbytes, C.byref(h)),
           "orkan_alloc_external")
    return h


def orkan_free(h):
    _check(_lib.orkan_free(h), "orkan_free")


def orkan_set_stream(h, stream_ptr: int | None):
    _check(_lib.orkan_set_stream(h, C.c_void_p(stream_ptr or 0)), "orkan_set_stream")


def orkan_set_fusion(h, max_ops: int, compose: bool = True):
    _check(_lib.orkan_set_fusion(h, max_ops, int(compose)), "orkan_set_fusion")


def orkan_get_info(h):
    v = [C.c_int() for _ in range(4)]
    _check(_lib.orkan_get_info(h, *[C.byref(x) for x in v]), "orkan_get_info")
    return tuple(x.value for x in v)


def orkan_autotune(n: int, dtype: int):
    """(tile_log2, max_ops) chosen by the library's autotuner for this device."""
    m, f = C.c_int(), C.c_int()
    _check(_lib.orkan_autotune(n, dtype, C.byref(m), C.byref(f)), "orkan_autotune")
    return m.value, f.value


def orkan_device_ptr(h) -> int:
    return int(_lib.orkan_device_ptr(h) or 0)


# ------------------------------------------------------------------ init
def orkan_init_state(h, kind: int, data=None):
    if data is None:
        _check(_lib.orkan_init_state(h, kind, None), "orkan_init_state")
        return
    arr = _cplx(data)
    _check(_lib.orkan_init_state(h, kind, _dptr(arr.view(np.float64))), "orkan_init_state")


def orkan_init_observable(h, paulis, coeffs):
    s = "".join(paulis).encode()
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    _check(_lib.orkan_init_observable(h, len(paulis), s, _dptr(c)), "orkan_init_observable")


def orkan_set_tensor(h, mode: int):
    _check(_lib.orkan_set_tensor(h, mode), "orkan_set_tensor")


def orkan_set_picture(h, picture: int):
    _check(_lib.orkan_set_picture(h, picture), "orkan_set_picture")


def orkan_load_tiled(h, host_buf: np.ndarray, picture: int = ORKAN_STATE):
    buf = np.ascontiguousarray(host_buf)
    _check(_lib.orkan_load_tiled(h, buf.ctypes.data_as(C.c_void_p), picture), "orkan_load_tiled")


def orkan_load_tiled_async(h, host_buf: np.ndarray, picture: int = ORKAN_STATE):
    """Queue the raw tiled upload on the handle's stream and return; host_buf
    (C-contiguous, ideally pinned) must stay alive and unchanged until the copy
    completes (orkan_sync or any blocking call on h)."""
    assert host_buf.flags["C_CONTIGUOUS"]
    _check(_lib.orkan_load_tiled_async(h, host_buf.ctypes.data_as(C.c_void_p), picture), "orkan_load_tiled_async")


def orkan_store_tiled(h, host_buf: np.ndarray):
    assert host_buf.flags["C_CONTIGUOUS"]
    _check(_lib.orkan_store_tiled(h, host_buf.ctypes.data_as(C.c_void_p)), "orkan_store_tiled")


def orkan_run_batch(items, stream_ptr=None):
    """Run an array of OrkanBatchItem in one call; returns the per-item
    statuses (ORKAN_OK, ORKAN_EZEROPROB, ORKAN_ETIMEOUT).  Validation errors
    raise OrkanError before anything runs."""
    arr = (OrkanBatchItem * len(items))(*items)
    st = _lib.orkan_run_batch(len(items), arr, C.c_void_p(stream_ptr or 0))
    statuses = [int(arr[i].status) for i in range(len(items))]
    if st != ORKAN_OK and not (st in (ORKAN_EZEROPROB, ORKAN_ETIMEOUT) and st in statuses):
        _check(st, "orkan_run_batch")
    return statuses


def orkan_batch_limits(max_ctas: int = 0, wait_seconds: float = 1.0):
    _check(_lib.orkan_batch_limits(max_ctas, wait_seconds), "orkan_batch_limits")


ORKAN_CKPT_HEADER_BYTES = 320


def orkan_checkpoint_save(h) -> np.ndarray:
    """The handle's checkpoint (header + raw tiled array) as a uint8 array."""
    buf = np.empty(int(_lib.orkan_checkpoint_bytes(h)), dtype=np.uint8)
    _check(_lib.orkan_checkpoint_save(h, buf.ctypes.data_as(C.c_void_p), buf.size), "orkan_checkpoint_save")
    return buf


def orkan_checkpoint_load(h, buf):
    buf = np.ascontiguousarray(np.frombuffer(buf, dtype=np.uint8) if not isinstance(buf, np.ndarray) else buf)
    _check(_lib.orkan_checkpoint_load(h, buf.ctypes.data_as(C.c_void_p), buf.nbytes), "orkan_checkpoint_load")


def orkan_checkpoint_inspect(buf) -> dict:
    """Header fields of a checkpoint after its checks (host only)."""
    buf = np.ascontiguousarray(np.frombuffer(buf, dtype=np.uint8) if not isinstance(buf, np.ndarray) else buf)
    n, dt, m, pic = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    _check(_lib.orkan_checkpoint_inspect(buf.ctypes.data_as(C.c_void_p), buf.nbytes, C.byref(n), C.byref(dt),
                                         C.byref(m), C.byref(pic)), "orkan_checkpoint_inspect")
    return {"n": n.value, "dtype": dt.value, "tile_log2": m.value, "picture": pic.value}


# ------------------------------------------------------------------ ops
def orkan_apply_unitary(h, qubits, U):
    k = len(qubits)
    M = _cplx(U)
    _check(_lib.orkan_apply_unitary(h, k, _qubits(qubits), _dptr(M.view(np.float64))), "orkan_apply_unitary")


def orkan_apply_kraus(h, qubits, kraus):
    k = len(qubits)
    K = _cplx(kraus, 1 << k)
    _check(_lib.orkan_apply_kraus(h, k, _qubits(qubits), K.shape[0], _dptr(K.view(np.float64))),
           "orkan_apply_kraus")


def orkan_depolarize(h, q: int, p: float):
    _check(_lib.orkan_depolarize(h, q, p), "orkan_depolarize")


def orkan_dephase(h, q: int, p: float):
    _check(_lib.orkan_dephase(h, q, p), "orkan_dephase")


def orkan_amplitude_damp(h, q: int, gamma: float):
    _check(_lib.orkan_amplitude_damp(h, q, gamma), "orkan_amplitude_damp")


def orkan_measure(h, q: int, u: float):
    out = C.c_int()
    prob = C.c_double()
    _check(_lib.orkan_measure(h, q, u, C.byref(out), C.byref(prob)), "orkan_measure")
    return out.value, prob.value


def orkan_project(h, q: int, outcome: int):
    _check(_lib.orkan_project(h, q, outcome), "orkan_project")


def orkan_run_circuit(h, ops_array, n_measure: int):
    """Apply a prepared OrkanOp array in one call; returns (outcomes, probs)."""
    outs = (C.c_int * max(n_measure, 1))()
    probs = (C.c_double * max(n_measure, 1))()
    done = C.c_int()
    _check(_lib.orkan_run_circuit(h, len(ops_array), ops_array, outs, probs, C.byref(done)), "orkan_run_circuit")
    return list(outs)[:n_measure], list(probs)[:n_measure]


# ------------------------------------------------------------------ readouts
def orkan_trace(h):
    re, im = C.c_double(), C.c_double()
    _check(_lib.orkan_trace(h, C.byref(re), C.byref(im)), "orkan_trace")
    return complex(re.value, im.value)


def orkan_expect_pauli(h, pauli: str) -> float:
    out = C.c_double()
    _check(_lib.orkan_expect_pauli(h, pauli.encode(), C.byref(out)), "orkan_expect_pauli")
    return out.value


def orkan_expect(rho, O) -> float:
    out = C.c_double()
    _check(_lib.orkan_expect(rho, O, C.byref(out)), "orkan_expect")
    return out.value


def orkan_to_dense(h) -> np.ndarray:
    n = orkan_get_info(h)[0]
    N = 1 << n
    out = np.empty((N, N), dtype=np.complex128)
    _check(_lib.orkan_to_dense(h, _dptr(out.view(np.float64))), "orkan_to_dense")
    return out


def orkan_get_elements(h, rows, cols) -> np.ndarray:
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    c = np.ascontiguousarray(np.asarray(cols, dtype=np.int64))
    assert r.shape == c.shape
    out = np.empty(r.size, dtype=np.complex128)
    _check(_lib.orkan_get_elements(h, r.size, r.ctypes.data_as(C.POINTER(_i64)), c.ctypes.data_as(C.POINTER(_i64)),
                                   _dptr(out.view(np.float64))), "orkan_get_elements")
    return out


def orkan_flush(h):
    _check(_lib.orkan_flush(h), "orkan_flush")


def orkan_sync(h):
    _check(_lib.orkan_sync(h), "orkan_sync")


def orkan_capture_begin(h):
    _check(_lib.orkan_capture_begin(h), "orkan_capture_begin")


def orkan_capture_end(h):
    g = C.c_void_p()
    _check(_lib.orkan_capture_end(h, C.byref(g)), "orkan_capture_end")
    return g


def orkan_graph_launch(h, graph):
    _check(_lib.orkan_graph_launch(h, graph), "orkan_graph_launch")


def orkan_graph_free(graph):
    _check(_lib.orkan_graph_free(graph), "orkan_graph_free")


def orkan_stats(h):
    v = [_i64() for _ in range(3)]
    _check(_lib.orkan_stats(h, *[C.byref(x) for x in v]), "orkan_stats")
    return {"passes": v[0].value, "ops": v[1].value, "launches": v[2].value}


def orkan_set_timing(h, enable: bool):
    _check(_lib.orkan_set_timing(h, int(enable)), "orkan_set_timing")


def orkan_pass_work(h):
    ops, nb = C.c_double(), C.c_double()
    _check(_lib.orkan_pass_work(h, C.byref(ops), C.byref(nb)), "orkan_pass_work")
    return ops.value, nb.value


ORKAN_NOALLOC_MAX_STRINGS = 64


def orkan_expect_paulis_noalloc(dev_state: int, n: int, dtype: int, tile_log2: int, paulis, stream_ptr=None):
    """tr(P_s H) for up to ORKAN_NOALLOC_MAX_STRINGS Pauli strings, read from a
    caller-owned tiled device array, with no device allocation (see orkan.h)."""
    out = np.zeros(len(paulis))
    s = "".join(paulis).encode()
    _check(_lib.orkan_expect_paulis_noalloc(C.c_void_p(dev_state), n, dtype, tile_log2, len(paulis), s, _dptr(out),
                                            C.c_void_p(stream_ptr or 0)), "orkan_expect_paulis_noalloc")
    return out


def orkan_probe_pipes(scratch_ptr: int, scratch_bytes: int) -> dict:
    """Measured pipe rates (instructions/s) and copy bandwidth (GB/s) of the current GPU."""
    out = (C.c_double * 6)()
    _check(_lib.orkan_probe_pipes(out, C.c_void_p(scratch_ptr), scratch_bytes), "orkan_probe_pipes")
    return {"fp32_fma_per_s": out[0], "fp64_fma_per_s": out[1], "fp32_add_per_s": out[2], "fp64_add_per_s": out[3],
            "copy_GBps": out[4], "fp32x2_fma_lanes_per_s": out[5]}


# ------------------------------------------------------------------ qubit relabelling
def orkan_relabel(h, phys):
    _check(_lib.orkan_relabel(h, _qubits(phys)), "orkan_relabel")


def orkan_get_labels(h, n: int):
    arr = (C.c_int * n)()
    _check(_lib.orkan_get_labels(h, arr), "orkan_get_labels")
    return list(arr)


def orkan_set_relabel(h, mode: int):
    _check(_lib.orkan_set_relabel(h, mode), "orkan_set_relabel")


# ------------------------------------------------------------------ packed column-major layout
def orkan_packed_bytes(n: int, dtype: int) -> int:
    return int(_lib.orkan_packed_bytes(n, dtype))


def orkan_packed_offset(n: int, i: int, j: int):
    cj = C.c_int()
    off = int(_lib.orkan_packed_offset(n, i, j, C.byref(cj)))
    return off, bool(cj.value)


def orkan_packed_apply_unitary(dev: int, n: int, dtype: int, qubits, U, picture=ORKAN_STATE, stream_ptr=None):
    M = _cplx(U)
    _check(_lib.orkan_packed_apply_unitary(C.c_void_p(dev), n, dtype, picture, len(qubits), _qubits(qubits),
                                           _dptr(M.view(np.float64)), C.c_void_p(stream_ptr or 0)),
           "orkan_packed_apply_unitary")


def orkan_packed_apply_kraus(dev: int, n: int, dtype: int, qubits, kraus, picture=ORKAN_STATE, stream_ptr=None):
    K = _cplx(kraus, 1 << len(qubits))
    _check(_lib.orkan_packed_apply_kraus(C.c_void_p(dev), n, dtype, picture, len(qubits), _qubits(qubits),
                                         K.shape[0], _dptr(K.view(np.float64)), C.c_void_p(stream_ptr or 0)),
           "orkan_packed_apply_kraus")


def orkan_packed_depolarize(dev: int, n: int, dtype: int, q: int, p: float, stream_ptr=None):
    _check(_lib.orkan_packed_depolarize(C.c_void_p(dev), n, dtype, q, p, C.c_void_p(stream_ptr or 0)),
           "orkan_packed_depolarize")


def orkan_packed_from_tiled(h, dev: int):
    _check(_lib.orkan_packed_from_tiled(h, C.c_void_p(dev)), "orkan_packed_from_tiled")


def orkan_packed_to_tiled(h, dev: int):
    _check(_lib.orkan_packed_to_tiled(h, C.c_void_p(dev)), "orkan_packed_to_tiled")


def orkan_pass_time(h):
    ms = C.c_double()
    cnt = _i64()
    _check(_lib.orkan_pass_time(h, C.byref(ms), C.byref(cnt)), "orkan_pass_time")
    return ms.value, cnt.value
