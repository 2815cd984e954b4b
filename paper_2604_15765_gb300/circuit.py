"""Issue an op list (the dicts of ``workloads.synth``) through the C ABI.

Marshalling only: every op becomes one call of the binding with the same
meaning; the library plans, fuses and runs the passes on the GPU.
"""
from __future__ import annotations

import numpy as np

from . import orkan as ok


def apply_op(h, op, picture: str = "schrodinger"):
    """Apply one op; returns (outcome, prob) for measurements, else None."""
    kind = op["kind"]
    q = op["qubits"]
    if kind == "unitary":
        ok.orkan_apply_unitary(h, q, op["matrix"])
    elif kind == "kraus":
        ok.orkan_apply_kraus(h, q, op["mats"])
    elif kind == "depolarize":
        ok.orkan_depolarize(h, q[0], op["p"])
    elif kind == "dephase":
        ok.orkan_dephase(h, q[0], op["p"])
    elif kind == "ampdamp":
        ok.orkan_amplitude_damp(h, q[0], op["gamma"])
    elif kind == "measure":
        if picture == "schrodinger":
            return ok.orkan_measure(h, q[0], op["u"])
        b = 0 if op["u"] < 0.5 else 1
        ok.orkan_project(h, q[0], b)
        return (b, None)
    elif kind == "project":
        ok.orkan_project(h, q[0], op["outcome"])
    else:
        raise ValueError(kind)
    return None


# orkan_op as a NumPy record (the ctypes structure's field offsets), so that an
# op list is marshalled with list appends and one record-array fill instead of
# per-field ctypes attribute writes
_OP_DTYPE = np.dtype({"names": ["kind", "k", "q0", "q1", "q2", "r", "outcome", "param", "mats"],
                      "formats": ["<i4", "<i4", "<i4", "<i4", "<i4", "<i4", "<i4", "<f8", "<u8"],
                      "offsets": [0, 4, 8, 12, 16, 20, 24, 32, 40], "itemsize": 48})
_KIND = {"unitary": ok.ORKAN_OP_UNITARY, "kraus": ok.ORKAN_OP_KRAUS, "depolarize": ok.ORKAN_OP_DEPOLARIZE,
         "dephase": ok.ORKAN_OP_DEPHASE, "ampdamp": ok.ORKAN_OP_AMPDAMP}


def marshal(ops, picture: str = "schrodinger"):
    """Op dicts -> (OrkanOp array, kept-alive buffers, number of MEASURE ops).
    On an observable a measurement becomes the projection b = (u >= 0.5)."""
    n = len(ops)
    kind, k, qs, r, outc, param, moff = [], [], [], [], [], [], []
    mats = []
    off = 0
    nmeas = 0
    for op in ops:
        kd = op["kind"]
        q = op["qubits"]
        k.append(len(q))
        qs.append((q + [0, 0, 0])[:3] if isinstance(q, list) else (list(q) + [0, 0, 0])[:3])
        o = 0
        pm = 0.0
        if kd == "unitary" or kd == "kraus":
            m = np.asarray(op["matrix"] if kd == "unitary" else op["mats"], np.complex128)
            mats.append(m.reshape(-1))
            r.append(1 if kd == "unitary" else m.shape[0])
            moff.append(off)
            off += m.size
            kind.append(_KIND[kd])
        else:
            r.append(0)
            moff.append(-1)
            if kd in ("depolarize", "dephase"):
                kind.append(_KIND[kd])
                pm = op["p"]
            elif kd == "ampdamp":
                kind.append(_KIND[kd])
                pm = op["gamma"]
            elif kd == "measure" and picture == "schrodinger":
                kind.append(ok.ORKAN_OP_MEASURE)
                pm = op["u"]
                nmeas += 1
            elif kd == "measure":
                kind.append(ok.ORKAN_OP_PROJECT)
                o = 0 if op["u"] < 0.5 else 1
            elif kd == "project":
                kind.append(ok.ORKAN_OP_PROJECT)
                o = op["outcome"]
            else:
                raise ValueError(kd)
        outc.append(o)
        param.append(pm)
    rec = np.zeros(max(n, 1), dtype=_OP_DTYPE)
    allm = np.ascontiguousarray(np.concatenate(mats)) if mats else np.zeros(1, np.complex128)
    if n:
        rec["kind"][:n] = kind
        rec["k"][:n] = k
        qa = np.asarray(qs, dtype=np.int32).reshape(n, 3)
        rec["q0"][:n], rec["q1"][:n], rec["q2"][:n] = qa[:, 0], qa[:, 1], qa[:, 2]
        rec["r"][:n] = r
        rec["outcome"][:n] = outc
        rec["param"][:n] = param
        mo = np.asarray(moff, dtype=np.int64)
        rec["mats"][:n] = np.where(mo >= 0, allm.ctypes.data + 16 * mo, 0).astype(np.uint64)
    arr = (ok.OrkanOp * max(n, 1)).from_buffer(rec)
    return arr, [rec, allm], nmeas


def run_circuit(h, ops, picture: str = "schrodinger", native: bool = True, marshalled=None):
    """Apply an op list; with native=True the whole list goes through one
    orkan_run_circuit call, else one binding call per op.  Returns the
    measurement records [(outcome, prob)] in order."""
    if not native:
        records = []
        for op in ops:
            rec = apply_op(h, op, picture)
            if rec is not None:
                records.append(rec)
        return records
    arr, keep, nmeas = marshalled if marshalled is not None else marshal(ops, picture)
    outs, probs = ok.orkan_run_circuit(h, arr, nmeas)
    del keep
    if picture == "schrodinger":
        return list(zip(outs, probs))
    return [(0 if op["u"] < 0.5 else 1, None) for op in ops if op["kind"] == "measure"]


def run_batch(requests, stream_ptr=None):
    """Marshal requests into one orkan_run_batch call.  Each request is a dict:
      h        handle; init: "pure" (psi0), "pauli_sum" (terms, coeffs) or "keep";
      ops      op dicts (measurements become projections on observables);
      paulis   readout strings (optional); psi: readout vector (optional);
      gang     CTAs (0 / absent = automatic).
    Returns one dict per request: out (tr(P H) per string, then <psi|H|psi>),
    outcomes, probs, status."""
    import numpy as np
    keep = []
    items = []
    outs = []
    for r in requests:
        it = ok.OrkanBatchItem()
        it.h = r["h"]
        init = r.get("init", "keep")
        picture = "heisenberg" if init == "pauli_sum" else "schrodinger"
        if init == "keep":
            it.init = ok.ORKAN_BATCH_KEEP
            picture = r.get("picture", "schrodinger")
        elif init == "pure":
            it.init = ok.ORKAN_INIT_PURE
            psi0 = np.ascontiguousarray(np.asarray(r["psi0"], np.complex128))
            keep.append(psi0)
            it.init_data = psi0.view(np.float64).ctypes.data_as(ok._pd)
        else:
            it.init = ok.ORKAN_BATCH_PAULI_SUM
            terms = "".join(r["terms"]).encode()
            cs = np.ascontiguousarray(np.asarray(r["coeffs"], np.float64))
            keep += [terms, cs]
            it.nterms = len(r["terms"])
            it.terms = terms
            it.coeffs = cs.ctypes.data_as(ok._pd)
        arr, kk, nmeas = r["marshalled"] if "marshalled" in r else marshal(r.get("ops", []), picture)
        keep += [arr, kk]
        it.nops = len(r.get("ops", []))
        it.ops = arr
        paulis = r.get("paulis", [])
        it.npaulis = len(paulis)
        if paulis:
            ps = "".join(paulis).encode()
            keep.append(ps)
            it.paulis = ps
        psi = r.get("psi")
        nout = len(paulis) + (0 if psi is None else 1)
        out = np.zeros(max(nout, 1))
        if psi is not None:
            pv = np.ascontiguousarray(np.asarray(psi, np.complex128))
            keep.append(pv)
            it.psi = pv.view(np.float64).ctypes.data_as(ok._pd)
        it.out = out.ctypes.data_as(ok._pd)
        oc = np.zeros(max(nmeas, 1), dtype=np.int32)
        pr = np.zeros(max(nmeas, 1))
        it.outcomes = oc.ctypes.data_as(ok._pi)
        it.probs = pr.ctypes.data_as(ok._pd)
        it.gang = int(r.get("gang", 0))
        outs.append((out, nout, oc, pr, nmeas))
        items.append(it)
    statuses = ok.orkan_run_batch(items, stream_ptr)
    del keep
    return [{"out": out[:nout].copy(), "outcomes": [int(x) for x in oc[:nm]], "probs": [float(x) for x in pr[:nm]],
             "status": s} for (out, nout, oc, pr, nm), s in zip(outs, statuses)]
