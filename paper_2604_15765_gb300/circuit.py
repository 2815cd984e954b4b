"""Issue an op list (the dicts of ``workloads.synth``) through the C ABI.

Marshalling only: every op becomes one call of the binding with the same
meaning; the library plans, fuses and runs the passes on the GPU.
"""
from __future__ import annotations

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


def marshal(ops, picture: str = "schrodinger"):
    """Op dicts -> (OrkanOp array, kept-alive matrices, number of MEASURE ops).
    On an observable a measurement becomes the projection b = (u >= 0.5)."""
    import numpy as np
    arr = (ok.OrkanOp * len(ops))()
    keep = []
    nmeas = 0
    for o, op in zip(arr, ops):
        kind = op["kind"]
        q = op["qubits"]
        o.k = len(q)
        for l in range(3):
            o.qubits[l] = q[l] if len(q) > l else 0
        if kind in ("unitary", "kraus"):
            mats = np.ascontiguousarray(np.asarray(op["matrix"] if kind == "unitary" else op["mats"], np.complex128))
            keep.append(mats)
            o.kind = ok.ORKAN_OP_UNITARY if kind == "unitary" else ok.ORKAN_OP_KRAUS
            o.r = 1 if kind == "unitary" else mats.shape[0]
            o.mats = mats.view(np.float64).ctypes.data_as(ok._pd)
        elif kind == "depolarize":
            o.kind, o.param = ok.ORKAN_OP_DEPOLARIZE, op["p"]
        elif kind == "dephase":
            o.kind, o.param = ok.ORKAN_OP_DEPHASE, op["p"]
        elif kind == "ampdamp":
            o.kind, o.param = ok.ORKAN_OP_AMPDAMP, op["gamma"]
        elif kind == "measure" and picture == "schrodinger":
            o.kind, o.param = ok.ORKAN_OP_MEASURE, op["u"]
            nmeas += 1
        elif kind == "measure":
            o.kind, o.outcome = ok.ORKAN_OP_PROJECT, 0 if op["u"] < 0.5 else 1
        elif kind == "project":
            o.kind, o.outcome = ok.ORKAN_OP_PROJECT, op["outcome"]
        else:
            raise ValueError(kind)
    return arr, keep, nmeas


def run_circuit(h, ops, picture: str = "schrodinger", native: bool = True):
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
    arr, keep, nmeas = marshal(ops, picture)
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
        arr, kk, nmeas = marshal(r.get("ops", []), picture)
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
