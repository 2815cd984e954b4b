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


def run_circuit(h, ops, picture: str = "schrodinger"):
    records = []
    for op in ops:
        rec = apply_op(h, op, picture)
        if rec is not None:
            records.append(rec)
    return records
