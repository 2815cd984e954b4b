#!/usr/bin/env python
"""k-local ops/s of the Orkan hot path on GB300 (one JSON line on stdout).

Workload (the per-op sweep at full size): an n = 14 operator in the tiled
lower-triangle layout (m = 5, 2.15 GB per operand at 16 B/element).  One step
is one pass of the whole hot path:

  Schroedinger, on a mixed state rho (Haar pure state depolarised on every
  qubit): for every target q a Haar 1-qubit U, depolarising p = 0.1 (4 Kraus),
  amplitude damping gamma = 0.05 (2 Kraus), a Haar 2-qubit U on (q, q+1) and
  on (q, n-1-q); then a Z measurement with a seeded draw, 8 Pauli-string
  expectations and the trace;
  Heisenberg, on a 16-term Pauli-sum observable O: the adjoint sweep in
  reverse order, then tr(rho O) from the tiled Frobenius products.

value = k-local ops (2 x 70 + 1 measurement per step) / device time, with the
operands resident in HBM and continuously evolved (as in Sec. IV-A), in
native FP64 arithmetic on complex128 storage (the paper's precision) unless
--dtype names another form.  The roofline is on the HBM basis (2 x stored
bytes per pass / average pass time / measured copy bandwidth) with the FP64
pipe's share of its derived peak beside it.  The line also carries the
first layers of the n = 16 noisy brickwork in FP64, the plain one-op-per-pass
FP64 path and the double-float and complex64 forms with their errors against
the FP64 run, single-op pass bandwidths, and a served sample with p50/p99.  e2e
repeats the step through the same C ABI with the operands uploaded from
pinned host memory every step and the scalars read back.  Under torchrun each
rank runs an independent replica (weak scaling, no collective on the data
path); value sums ops over ranks and divides by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "k-local ops/s & HBM % peak, plain FP64 vs served/batched/FP32 forms; p50/p99"
UNIT = "ops/s"
DTYPE_NAMES = {"c128": 0, "c64": 1, "df64": 2}


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["orkan", "reference"], default="orkan")
    p.add_argument("--dtype", choices=list(DTYPE_NAMES), default="c128")
    p.add_argument("--n", type=int, default=14)
    p.add_argument("--tile-log2", type=int, default=5)
    p.add_argument("--fusion", type=int, default=8)
    p.add_argument("--no-compose", action="store_true")
    p.add_argument("--no-variants", action="store_true", help="skip the c128 / c64 / unfused comparison runs")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=20.0)
    p.add_argument("--workload", choices=["sweep", "serving", "brickwork", "precision", "paper", "relabel", "pipes",
                                          "tensor", "batch"],
                   default="sweep")
    p.add_argument("--depth", type=int, default=40)
    p.add_argument("--bw-depth", type=int, default=6,
                   help="layers of the n=16 noisy brickwork timed in the default run (0 = skip)")
    p.add_argument("--serve-requests", type=int, default=160,
                   help="requests in the serving sample of the default run (the serving workload uses 5000)")
    p.add_argument("--paper-sizes", default="6,8,10,12,13,14,15,16", help="qubit counts of the paper study")
    p.add_argument("--paper-ops", default="depolarize,x,hadamard,cnot", help="experiments of the paper study")
    p.add_argument("--paper-dtypes", default="c128,df64", help="storage types of the paper study")
    p.add_argument("--paper-layouts", default="packed,tiled,tiled_fused", help="layouts of the paper study")
    p.add_argument("--op-class", default=None,
                   help="time only single-op passes of one class (u1_in, u2_in_cross, ...) and print their GB/s")
    return p.parse_args(argv)


# ------------------------------------------------------------------ distributed plumbing
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(units: float, seconds: float, group=None):
    """Whole-job throughput: sum of units over ranks / max of seconds over ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return units, seconds
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    s = torch.tensor([float(seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(s, op=dist.ReduceOp.MAX, group=group)
    return float(u.item()), float(s.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ------------------------------------------------------------------ host placement
def parse_cpulist(spec: str) -> set:
    """The CPU set of a Linux cpulist string such as "0-3,8,10-11"."""
    cpus = set()
    for part in spec.strip().split(","):
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif part:
            cpus.add(int(part))
    return cpus


def bind_near_gpu(torch, dev: int):
    """Run this process on the CPU cores local to the GPU (its PCI device's
    local_cpulist), so that pinned host buffers are first touched on the NUMA
    node the GPU is attached to.  Returns the bound core count, or None when
    the topology is not exposed."""
    try:
        pr = torch.cuda.get_device_properties(dev)
        bdf = f"{int(pr.pci_domain_id):04x}:{int(pr.pci_bus_id):02x}:{int(pr.pci_device_id):02x}.0"
        with open(f"/sys/bus/pci/devices/{bdf}/local_cpulist") as f:
            cpus = parse_cpulist(f.read())
        cpus &= os.sched_getaffinity(0)
        if not cpus:
            return None
        os.sched_setaffinity(0, cpus)
        return len(cpus)
    except (AttributeError, OSError, ValueError):
        return None


# ------------------------------------------------------------------ clocks
def gpu_uuid(torch, local: int) -> str:
    """nvidia-smi id of the current device (its UUID, else the local index)."""
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    except Exception:  # noqa: BLE001  (older torch without uuid)
        return str(local)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu = gpu_id
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.remove(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        loaded = sorted(sm)[len(sm) // 2:] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ workload
def make_workload(n: int):
    from workloads import synth as S
    rng = S.rng_for(S.BASE_SEED + 1)
    ops = S.sweep(n)
    psi = S.haar_state_vector(rng, 1 << n)
    paulis = S.random_pauli_strings(rng, n, 8)
    obs_strings, obs_coeffs = S.random_pauli_sum(rng, n, 16)
    us = rng.uniform(0.0, 1.0, 64)
    return {"ops": ops, "psi": psi, "paulis": paulis, "obs": (obs_strings, obs_coeffs), "us": us}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# Derived ALU peaks: the device's SM count x the pipe's unit rate per SM per clock x the 2070 MHz maximum
# SM clock.  Unit rates: FP32 128 lanes (4 x 32 FP32 units; the pipe probe measures 119-125), FP64 2 operations
# (the pipe probe measures 1.97 FMA per SM per clock on GB300).
UNIT_RATE = {"df64": 128.0, "c64": 128.0, "c128": 2.0}
SM_MAX_HZ = 2.07e9


def alu_peak_tops(dtype: str, sms: int) -> float:
    return sms * UNIT_RATE[dtype] * SM_MAX_HZ / 1e12


PASS_SOURCES = ("pass_kernels.cuh", "numeric.cuh", "device_util.cuh")


def pass_source_digest() -> str:
    """First 16 hex digits of the SHA-256 of the pass kernel's device sources,
    concatenated in PASS_SOURCES order."""
    h = hashlib.sha256()
    for name in PASS_SOURCES:
        with open(os.path.join(ROOT, "paper_2604_15765_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_record(dtype: str):
    """DRAM bytes per pass-kernel launch from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "pass_kernel_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        digest = pass_source_digest()
        ent = rec.get(dtype)
        if ent and ent.get("source_sha256_16") == digest:
            return ent
    except (OSError, ValueError):
        pass
    return None


class Runner:
    """Two handles (rho, O) on one stream, the sweep issued through the C ABI."""

    def __init__(self, ok, circuit, wl, n, m, dtype, fusion, compose, stream):
        self.ok, self.circuit, self.wl = ok, circuit, wl
        self.n = n
        self.rho = ok.orkan_alloc(n, DTYPE_NAMES[dtype], m)
        self.O = ok.orkan_alloc(n, DTYPE_NAMES[dtype], m)
        for h in (self.rho, self.O):
            ok.orkan_set_stream(h, stream)
            ok.orkan_set_fusion(h, fusion, compose)
        ok.orkan_init_state(self.rho, ok.ORKAN_INIT_PURE, wl["psi"])
        for q in range(n):
            ok.orkan_depolarize(self.rho, q, 0.1)
        ok.orkan_init_observable(self.O, *wl["obs"])
        ok.orkan_sync(self.rho)
        self.bytes = ok.orkan_bytes(n, DTYPE_NAMES[dtype], m)
        self.step_idx = 0
        self.ops_per_step = 2 * len(wl["ops"]) + 1
        # the sweep marshalled once into C-ABI op arrays (one orkan_run_circuit call per picture)
        self.sch = circuit.marshal(wl["ops"], "schrodinger")
        self.hei = circuit.marshal(list(reversed(wl["ops"])), "heisenberg")

    def step(self):
        ok, wl = self.ok, self.wl
        ok.orkan_run_circuit(self.rho, self.sch[0], 0)
        q = self.step_idx % self.n
        u = float(wl["us"][self.step_idx % len(wl["us"])])
        res = [ok.orkan_measure(self.rho, q, u)[1]]
        res += [ok.orkan_expect_pauli(self.rho, s) for s in wl["paulis"]]
        res.append(ok.orkan_trace(self.rho).real)
        ok.orkan_run_circuit(self.O, self.hei[0], 0)
        res.append(ok.orkan_expect(self.rho, self.O))
        self.step_idx += 1
        return res

    def launches(self):
        return sum(self.ok.orkan_stats(h)["launches"] for h in (self.rho, self.O))

    def timing(self, enable):
        for h in (self.rho, self.O):
            self.ok.orkan_set_timing(h, enable)

    def pass_time(self):
        ms, cnt = 0.0, 0
        self.work = [0.0, 0.0]
        for h in (self.rho, self.O):
            w = self.ok.orkan_pass_work(h)
            self.work[0] += w[0]
            self.work[1] += w[1]
            a, b = self.ok.orkan_pass_time(h)
            ms += a
            cnt += b
        return ms, cnt

    def free(self):
        self.ok.orkan_free(self.rho)
        self.ok.orkan_free(self.O)


def per_op_table(ok, wl, n, m, dtypes, stream, torch, reps=4, only=None):
    """HBM GB/s of single-op passes (fusion 1, no composition) per op class,
    in-tile (target 1 < m) and cross-tile (target n-2 >= m), per dtype: the
    per-pass view of the sweep (2 x stored bytes / pass time).  Three-qubit
    classes run the block-update kernel (all targets in-tile, all three
    cross-tile, mixed; a Toffoli as the monomial form).  Beside it, the
    achieved algorithmic ALU rate (Tops/s) of the classes that do arithmetic."""
    from workloads import synth as S
    rng = S.rng_for(S.BASE_SEED + 11)
    U1, U2, U3 = S.haar_unitary(rng, 2), S.haar_unitary(rng, 4), S.haar_unitary(rng, 8)
    toffoli = np.zeros((8, 8), dtype=np.complex128)
    for b in range(8):
        toffoli[b ^ (4 if (b & 3) == 3 else 0), b] = 1
    xg = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    cnot = np.eye(4, dtype=np.complex128)[[0, 3, 2, 1]]
    lo, hi = 1, n - 2
    classes = {
        "u1_in": lambda h: ok.orkan_apply_unitary(h, [lo], U1),
        "u1_cross": lambda h: ok.orkan_apply_unitary(h, [hi], U1),
        "depol_in": lambda h: ok.orkan_depolarize(h, lo, 0.1),
        "depol_cross": lambda h: ok.orkan_depolarize(h, hi, 0.1),
        "ampdamp_in": lambda h: ok.orkan_amplitude_damp(h, lo, 0.05),
        "ampdamp_cross": lambda h: ok.orkan_amplitude_damp(h, hi, 0.05),
        "u2_in_in": lambda h: ok.orkan_apply_unitary(h, [lo, lo + 1], U2),
        "u2_in_cross": lambda h: ok.orkan_apply_unitary(h, [lo, hi], U2),
        "u2_cross_cross": lambda h: ok.orkan_apply_unitary(h, [hi - 1, hi], U2),
        "x_in": lambda h: ok.orkan_apply_unitary(h, [lo], xg),
        "x_cross": lambda h: ok.orkan_apply_unitary(h, [hi], xg),
        "cnot_in_cross": lambda h: ok.orkan_apply_unitary(h, [lo, hi], cnot),
        "cnot_cross_cross": lambda h: ok.orkan_apply_unitary(h, [hi, hi - 1], cnot),
        "u3_in": lambda h: ok.orkan_apply_unitary(h, [0, 1, 2], U3),
        "u3_mixed": lambda h: ok.orkan_apply_unitary(h, [lo, n // 2, n - 1], U3),
        "u3_cross": lambda h: ok.orkan_apply_unitary(h, [n - 3, n - 2, n - 1], U3),
        "toffoli_cross": lambda h: ok.orkan_apply_unitary(h, [n - 1, n - 2, lo], toffoli),
    }
    if only is not None:
        classes = {only: classes[only]}
    out = {}
    for dt in dtypes:
        h = ok.orkan_alloc(n, DTYPE_NAMES[dt], m)
        ok.orkan_set_stream(h, stream)
        ok.orkan_set_fusion(h, 1, False)
        ok.orkan_init_state(h, ok.ORKAN_INIT_PURE, wl["psi"])
        nbytes = 2 * ok.orkan_bytes(n, DTYPE_NAMES[dt], m)
        row, alu = {}, {}
        for name, fn in classes.items():
            fn(h)
            ok.orkan_sync(h)
            ok.orkan_set_timing(h, True)
            ok.orkan_pass_time(h)
            ok.orkan_pass_work(h)
            for _ in range(reps):
                fn(h)
            ms, cnt = ok.orkan_pass_time(h)
            work, _ = ok.orkan_pass_work(h)
            ok.orkan_set_timing(h, False)
            row[name] = round(nbytes / (ms / cnt * 1e-3) / 1e9, 1)
            if work > 0:
                alu[name] = round(work / (ms * 1e-3) / 1e12, 2)
        out[dt] = row
        out[dt + "_alu_Tops"] = alu
        ok.orkan_free(h)
    return out


def _request_errors(reqs, res, ref):
    """Largest |result - reference| per request dtype (c128 / c64 requests)."""
    out = {}
    for dt in ("c128", "c64"):
        d = [float(np.max(np.abs(np.asarray(res[r["id"]]) - np.asarray(ref[r["id"]])))) for r in reqs
             if r["dtype"] == dt and r["id"] in res and r["id"] in ref]
        out[f"max_abs_err_{dt}_requests"] = max(d) if d else None
    return out


def tensor_study(ok, circuit, n, m, stream, reps=5):
    """complex64 in-tile runs of 1, 2, 4 and 8 Haar two-qubit unitaries on the
    tile's qubits: the CUDA-core fused pass (orkan_set_tensor 0) against the
    tensor-core pass of the composed block (mode 2); time per run and the
    passes' HBM rate (2 x stored bytes / pass time)."""
    from workloads import synth as S
    rng = S.rng_for(S.BASE_SEED + 15)
    psi = S.haar_state_vector(rng, 1 << n)
    nb = 2 * ok.orkan_bytes(n, ok.ORKAN_C64, m)
    out = {"n": n, "dtype": "c64", "tile_log2": m}
    for count in (1, 2, 4, 8):
        ops = []
        for _ in range(count):
            a, b = rng.choice(m, size=2, replace=False)
            ops.append(S.op_unitary(S.haar_unitary(rng, 4), [int(a), int(b)]))
        row = {}
        for label, mode in (("cuda_cores", 0), ("tensor_cores", 2)):
            h = ok.orkan_alloc(n, ok.ORKAN_C64, m)
            ok.orkan_set_stream(h, stream)
            ok.orkan_set_fusion(h, 16, True)
            ok.orkan_set_tensor(h, mode)
            ok.orkan_init_state(h, ok.ORKAN_INIT_PURE, psi)
            circuit.run_circuit(h, ops)
            ok.orkan_sync(h)
            ok.orkan_set_timing(h, True)
            ok.orkan_pass_time(h)
            for _ in range(reps):
                circuit.run_circuit(h, ops)
                ok.orkan_flush(h)
            ms, cnt = ok.orkan_pass_time(h)
            ok.orkan_free(h)
            row[label] = {"ms_per_run": round(ms / reps, 4), "passes_per_run": cnt / reps,
                          "pass_GBps": round(nb / (ms / cnt * 1e-3) / 1e9, 1)}
        row["speedup"] = round(row["cuda_cores"]["ms_per_run"] / row["tensor_cores"]["ms_per_run"], 2)
        out[f"u2_x{count}"] = row
    return out


def serving_study(reqs, torch, budget, slots=8, realtime_fracs=(0.8,), baseline=True, batch_max_n=8):
    """Continuous batching vs one-at-a-time plain FP64 on the same requests.
    The plain arm runs every request alone, one pass per op, in native FP64
    (c64 requests too); its results are the reference for every served arm's
    per-request error.  Served arms: requests at their own dtype (c128 in
    native FP64, c64 in FP32) and, separately, c128 requests in double-float.
    Capacity: all requests present at t = 0; latency runs: Poisson arrivals at
    a fraction of the measured capacity (arrival times rescaled), served in
    arrival order (fifo) and shortest-estimated-work first (sjf)."""
    from paper_2604_15765_gb300 import serving
    serving.prepare(reqs)   # circuits arrive as C-ABI op arrays (marshalled before timing)
    out = {"requests": len(reqs), "slots": slots, "memory_budget_bytes": budget,
           "served_form": f"{slots} concurrent slots, fused passes (8 ops, composed); *_batched: requests of "
                          f"n <= {batch_max_n} in persistent batched launches (orkan_run_batch) beside the slots; "
                          "latency runs on the c128 batched form"}
    ref = None
    if baseline:
        ref, b = serving.serve(reqs, budget, slots=1, dtype_map={"c64": "c128"}, fusion=1, compose=False,
                               realtime=False)
        out["plain_fp64_one_at_a_time"] = b
    arms = (("c128", {}, None), ("c128_batched", {}, batch_max_n), ("df64", {"c128": "df64"}, None),
            ("df64_batched", {"c128": "df64"}, batch_max_n))
    cap = None
    for label, dmap, bmax in arms:
        res, st = serving.serve(reqs, budget, slots=slots, dtype_map=dmap, realtime=False, batch_max_n=bmax)
        st["c128_requests_in"] = label.split("_")[0]
        if ref is not None:
            st.update(_request_errors(reqs, res, ref))
        out[f"served_capacity_{label}"] = st
        if label == "c128_batched":
            cap = st
    out["served_capacity"] = cap
    base_t = [r["t"] for r in reqs]
    for frac in realtime_fracs:
        rate = frac * cap["solves_per_s"]
        span = base_t[-1] if base_t[-1] > 0 else 1.0
        scaled = [dict(r, t=r["t"] * (len(reqs) / rate) / span) for r in reqs]
        _, st = serving.serve(scaled, budget, slots=slots, realtime=True, batch_max_n=batch_max_n)
        out[f"served_at_{frac:.1f}x_capacity"] = st
        _, st = serving.serve(scaled, budget, slots=slots, realtime=True, policy="sjf", batch_max_n=batch_max_n)
        out[f"served_at_{frac:.1f}x_capacity_sjf"] = st
    torch.cuda.synchronize()
    return out


def _run_timed(ok, circuit, torch, stream, n, dt, m, fusion, compose, ops, paulis, psi):
    """One operator through ops, then the Pauli strings; device time, pass stats, handle."""
    h = ok.orkan_alloc(n, DTYPE_NAMES[dt], m)
    ok.orkan_set_stream(h, stream)
    ok.orkan_set_fusion(h, fusion, compose)
    ok.orkan_init_state(h, ok.ORKAN_INIT_PURE, psi)
    ok.orkan_sync(h)
    ok.orkan_set_timing(h, True)
    ok.orkan_pass_time(h)
    ok.orkan_pass_work(h)
    p0 = ok.orkan_stats(h)["passes"]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for op in ops:
        circuit.apply_op(h, op)
    ok.orkan_flush(h)
    ev1.record()
    exps = np.array([ok.orkan_expect_pauli(h, s) for s in paulis])
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    pass_ms, cnt = ok.orkan_pass_time(h)
    work, _ = ok.orkan_pass_work(h)
    ok.orkan_set_timing(h, False)
    nb = 2 * ok.orkan_bytes(n, DTYPE_NAMES[dt], m)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    st = {"ops_per_s": round(len(ops) / (ms / 1e3), 1), "ms": round(ms, 1), "passes": ok.orkan_stats(h)["passes"] - p0,
          "tile_log2": m, "fusion": fusion, "compose": compose,
          "avg_pass_GBps": round(nb / (pass_ms / max(cnt, 1) * 1e-3) / 1e9, 1),
          "avg_pass_hbm_frac": round(nb / (pass_ms / max(cnt, 1) * 1e-3) / 1e9 / peaks()[0], 4),
          "pass_share": round(pass_ms / ms, 4) if ms > 0 else None,
          ("fp64_pipe_frac" if dt == "c128" else "fp32_pipe_frac"):
              round(work / (pass_ms * 1e-3) / 1e12 / alu_peak_tops(dt, sms), 4) if pass_ms > 0 else None,
          "trace_error": abs(ok.orkan_trace(h) - 1.0)}
    return h, st, exps


def small_request_study(S, torch, count=600, budget=8 << 30):
    """Requests of n = 4..10 (the serving mix's small end, where every op is
    launch-bound): solves/s with the slots alone, and with the batched
    persistent launch for n <= 8 beside them; same requests, own dtypes."""
    from paper_2604_15765_gb300 import serving
    reqs = serving.prepare(S.serving_stream(count=count, seed=S.BASE_SEED + 14, n_range=(4, 10)))
    out = {"requests": count, "n_range": [4, 10]}
    res = {}
    for label, bmax in (("slots_only", None), ("batched_n_le_8", 8)):
        res[label], st = serving.serve(reqs, budget, slots=8, realtime=False, batch_max_n=bmax)
        out[label] = {k: (round(v, 3) if isinstance(v, float) else v) for k, v in st.items()}
    out.update({"batched_" + k: v for k, v in _request_errors(reqs, res["batched_n_le_8"], res["slots_only"]).items()})
    out["speedup_solves_per_s"] = round(out["batched_n_le_8"]["solves_per_s"] / out["slots_only"]["solves_per_s"], 2)
    torch.cuda.synchronize()
    return out


def sweep_elements(ok, circuit, wl, n, m, dt, fusion, compose, stream, sample=None):
    """One Schroedinger sweep from the bench's initial state (the Haar pure
    state depolarised on every qubit) in the given form; returns sampled
    elements (complex128) and the sample (rows, cols, diagonal count)."""
    h = ok.orkan_alloc(n, DTYPE_NAMES[dt], m)
    ok.orkan_set_stream(h, stream)
    ok.orkan_set_fusion(h, fusion, compose)
    ok.orkan_init_state(h, ok.ORKAN_INIT_PURE, wl["psi"])
    for q in range(n):
        ok.orkan_depolarize(h, q, 0.1)
    arr, keep, _ = circuit.marshal(wl["ops"], "schrodinger")
    ok.orkan_run_circuit(h, arr, 0)
    if sample is None:
        rng = np.random.Generator(np.random.PCG64(20260415 + 21))
        N = 1 << n
        d = rng.integers(0, N, 4096)
        rows = np.concatenate([rng.integers(0, N, 1 << 16), d])
        cols = np.concatenate([rng.integers(0, N, 1 << 16), d])
        sample = (rows, cols, d.size)
    got = ok.orkan_get_elements(h, sample[0], sample[1])
    ok.orkan_free(h)
    del keep
    return got, sample


def brickwork_prefix(ok, circuit, torch, stream, n, dt, depth, hbm_peak):
    """The first `depth` layers of the config-2 noisy brickwork (n = 16, Haar
    1q on all qubits, Haar 2q on alternating pairs, depolarising 1e-3 on all)
    in the given form, tile m = 5, fusion 8 with composition: ops/s and the
    per-pass HBM fraction (2 x stored bytes / average pass time / hbm_gbs).
    Every layer has the same op mix, so a prefix has the full circuit's
    per-pass figures; `--workload brickwork` runs all 40 layers."""
    from workloads import synth as S
    rng = S.rng_for(S.BASE_SEED + 2)
    psi = S.haar_state_vector(rng, 1 << n)
    paulis = S.random_pauli_strings(rng, n, 32)
    ops = S.brickwork(n, depth)
    h, st, ex = _run_timed(ok, circuit, torch, stream, n, dt, 5, 8, True, ops, paulis, psi)
    ok.orkan_free(h)
    torch.cuda.empty_cache()
    st.update({"n": n, "dtype": dt, "layers": depth, "ops": len(ops),
               "state_bytes": ok.orkan_bytes(n, DTYPE_NAMES[dt], 5),
               "pauli_expectations_abs_max": float(np.max(np.abs(ex))),
               "workload": f"noisy brickwork n={n}, first {depth} of 40 layers (config 2), m=5, fusion 8 composed"})
    return st


def brickwork_study(ok, circuit, torch, stream, n, dt, depth):
    """Layered noisy brickwork (Haar 1q on all qubits, Haar 2q on alternating
    pairs, depolarising 1e-3 on all), autotuned tile size and fusion depth
    against the unfused schedule (m = 5, one pass per op), 32 Pauli strings."""
    from workloads import synth as S
    rng = S.rng_for(S.BASE_SEED + 2)
    psi = S.haar_state_vector(rng, 1 << n)
    paulis = S.random_pauli_strings(rng, n, 32)
    ops = S.brickwork(n, depth)
    t0 = time.perf_counter()
    m, f = ok.orkan_autotune(n, DTYPE_NAMES[dt])
    tune_s = time.perf_counter() - t0
    out = {"n": n, "dtype": dt, "depth": depth, "ops": len(ops), "autotune_s": round(tune_s, 2)}
    res = {}
    for label, (mm, ff, cc) in (("autotuned", (m, f, True)), ("unfused", (5, 1, False))):
        h, st, ex = _run_timed(ok, circuit, torch, stream, n, dt, mm, ff, cc, ops, paulis, psi)
        ok.orkan_free(h)
        out[label] = st
        res[label] = ex
    out["max_expectation_diff_tuned_vs_unfused"] = float(np.max(np.abs(res["autotuned"] - res["unfused"])))
    out["speedup_tuned_over_unfused"] = round(out["autotuned"]["ops_per_s"] / out["unfused"]["ops_per_s"], 2)
    return out


def paper_study(ok, torch, stream, dtypes=("c128", "df64"), ns=(6, 8, 10, 12, 13, 14, 15, 16), min_ms=40.0,
                experiments=("depolarize", "x", "hadamard", "cnot"), layouts=("packed", "tiled", "tiled_fused")):
    """The paper's own experiments (Sec. IV and its appendix): the depolarising
    channel with p = 0.1, Pauli X, Hadamard and CNOT; time per execution
    averaged over all qubit positions (all ordered pairs for CNOT), a layer
    applying the op at every position in turn to a continuously evolved random
    hermitian operator (a 16-term Pauli sum: neither positive nor normalised),
    after one warm-up layer.  Layouts: packed column-major and tiled (m = 5)
    with one op per pass -- the paper's comparison -- and tiled with fusion
    (8 ops, composition).  Effective bandwidth as the paper defines it: stored
    bytes / time per op, in GiB/s."""
    from workloads import synth as S
    had = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2)
    xg = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    cnot = np.eye(4, dtype=np.complex128)[[0, 3, 2, 1]]
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    cur = torch.cuda.current_stream()

    def timed(layer):
        layer()                                   # warm-up layer
        cur.synchronize()
        reps = 1
        while True:
            ev[0].record(cur)
            for _ in range(reps):
                layer()
            ev[1].record(cur)
            ev[1].synchronize()
            ms = ev[0].elapsed_time(ev[1])
            if ms >= min_ms or reps >= 64:
                return ms / reps
            reps = min(64, max(2 * reps, int(reps * min_ms / max(ms, 1e-3)) + 1))

    out = {}
    for dt in dtypes:
        code = DTYPE_NAMES[dt]
        table = {}
        for n in ns:
            rng = S.rng_for(S.BASE_SEED + 12 + n)
            strings, coeffs = S.random_pauli_sum(rng, n, 16)
            pos1 = [[q] for q in range(n)]
            pos2 = [[c, t] for c in range(n) for t in range(n) if c != t]
            cases = {k: v for k, v in {"depolarize": pos1, "x": pos1, "hadamard": pos1, "cnot": pos2}.items()
                     if k in experiments}
            ht = ok.orkan_alloc(n, code, 5)
            buf = torch.empty(ok.orkan_packed_bytes(n, code), dtype=torch.uint8, device="cuda")
            ok.orkan_set_stream(ht, stream)
            ok.orkan_init_observable(ht, strings, coeffs)
            ok.orkan_set_picture(ht, ok.ORKAN_STATE)
            ok.orkan_packed_from_tiled(ht, buf.data_ptr())   # both layouts start from the same operator
            dev = buf.data_ptr()
            tiled_bytes = ok.orkan_bytes(n, code, 5)
            packed_bytes = ok.orkan_packed_bytes(n, code)
            row = {"tiled_bytes": tiled_bytes, "packed_bytes": packed_bytes}
            for name, pos in cases.items():
                def tiled_layer(f, c, pos=pos, name=name):
                    ok.orkan_set_fusion(ht, f, c)
                    for q in pos:
                        if name == "depolarize":
                            ok.orkan_depolarize(ht, q[0], 0.1)
                        else:
                            ok.orkan_apply_unitary(ht, q, {"x": xg, "hadamard": had, "cnot": cnot}[name])
                    ok.orkan_flush(ht)

                def packed_layer(pos=pos, name=name):
                    for q in pos:
                        if name == "depolarize":
                            ok.orkan_packed_depolarize(dev, n, code, q[0], 0.1, stream)
                        else:
                            ok.orkan_packed_apply_unitary(dev, n, code, q, {"x": xg, "hadamard": had, "cnot": cnot}[name],
                                                          ok.ORKAN_STATE, stream)
                res = {}
                for label, fn, nbytes in (("packed", packed_layer, packed_bytes),
                                          ("tiled", lambda: tiled_layer(1, False), tiled_bytes),
                                          ("tiled_fused", lambda: tiled_layer(8, True), tiled_bytes)):
                    if label not in layouts:
                        continue
                    us = timed(fn) * 1e3 / len(pos)
                    res[label + "_us"] = round(us, 3)
                    res[label + "_GiBps"] = round(nbytes / (us * 1e-6) / 2 ** 30, 1)
                if "packed_us" in res and "tiled_us" in res:
                    res["tiled_speedup_over_packed"] = round(res["packed_us"] / res["tiled_us"], 3)
                row[name] = res
            ok.orkan_free(ht)
            del buf
            torch.cuda.empty_cache()
            table[str(n)] = row
        out[dt] = table
    return out


def relabel_study(ok, circuit, torch, stream, n=16, depth=40, dtypes=("df64", "c64")):
    """Qubit relabelling on a circuit concentrated on the five highest qubits
    (Haar 1q on each, Haar 2q on alternating neighbour pairs, depolarising
    1e-3 on each, per layer): automatic relabelling (the hot qubits swapped
    into the tile first) against none; same fusion (8 ops, composition)."""
    from workloads import synth as S
    rng = S.rng_for(S.BASE_SEED + 13)
    hot = list(range(n - 5, n))
    ops = []
    for layer in range(depth):
        for q in hot:
            ops.append(S.op_unitary(S.haar_unitary(rng, 2), [q]))
        for a in range(layer % 2, 4, 2):
            ops.append(S.op_unitary(S.haar_unitary(rng, 4), [hot[a], hot[a + 1]]))
        for q in hot:
            ops.append(S.op_depolarize(q, 1e-3))
    psi = S.haar_state_vector(rng, 1 << n)
    paulis = S.random_pauli_strings(rng, n, 8)
    arr, keep, _ = circuit.marshal(ops)
    out = {"n": n, "depth": depth, "ops": len(ops), "hot_qubits": hot}
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    cur = torch.cuda.current_stream()
    for dt in dtypes:
        row, res = {}, {}
        for mode in (0, 1):
            h = ok.orkan_alloc(n, DTYPE_NAMES[dt], 5)
            ok.orkan_set_stream(h, stream)
            ok.orkan_set_fusion(h, 8, True)
            ok.orkan_set_relabel(h, mode)
            ok.orkan_init_state(h, ok.ORKAN_INIT_PURE, psi)
            ok.orkan_sync(h)
            p0 = ok.orkan_stats(h)["passes"]
            ev[0].record(cur)
            ok.orkan_run_circuit(h, arr, 0)
            ok.orkan_flush(h)
            ev[1].record(cur)
            ev[1].synchronize()
            ms = ev[0].elapsed_time(ev[1])
            passes = ok.orkan_stats(h)["passes"] - p0
            res[mode] = np.array([ok.orkan_expect_pauli(h, s) for s in paulis])
            row["relabel" if mode else "plain"] = {"ms": round(ms, 2), "ops_per_s": round(len(ops) / (ms * 1e-3), 1),
                                                   "passes": passes, "labels_after": ok.orkan_get_labels(h, n)}
            ok.orkan_free(h)
        row["speedup"] = round(row["plain"]["ms"] / row["relabel"]["ms"], 3)
        row["max_expectation_diff"] = float(np.max(np.abs(res[0] - res[1])))
        out[dt] = row
    del keep
    return out


def precision_study(ok, circuit, torch, stream, depth):
    """Trace distance / max |delta| / Frobenius / trace error of the storage
    and arithmetic forms on the depth-40 noisy brickwork: against the CPU
    oracle at n = 10, against the GPU complex128 run at n = 12 and n = 16, and
    against the GPU double-float run at n = 17 (complex64 only otherwise)."""
    from oracle import dense as D
    from workloads import synth as S
    out = {}

    def states(n, dts, m=5):
        rng = S.rng_for(S.BASE_SEED + 3)
        psi = S.haar_state_vector(rng, 1 << n)
        ops = S.brickwork(n, depth, seed=S.BASE_SEED + 3)
        return psi, ops

    # n = 10: every form against the oracle (dense, CPU)
    n = 10
    psi, ops = states(n, None)
    t0 = time.perf_counter()
    ref, _ = D.run_circuit(np.outer(psi, psi.conj()), ops)
    cpu_s = time.perf_counter() - t0
    row = {"oracle_cpu_s": round(cpu_s, 1)}
    for dt in ("c128", "df64", "c64"):
        h, st, _ = _run_timed(ok, circuit, torch, stream, n, dt, 5, 8, True, ops, [], psi)
        got = ok.orkan_to_dense(h)
        ok.orkan_free(h)
        row[dt] = {"max_abs": D.max_abs_diff(got, ref), "frobenius": D.frobenius_diff(got, ref),
                   "trace_distance": D.trace_distance(got, ref), "trace_error": st["trace_error"]}
    out["n10_vs_oracle"] = row
    # n = 12: df64 and c64 against the GPU complex128 run (dense download, exact trace distance)
    n = 12
    psi, ops = states(n, None)
    dense = {}
    for dt in ("c128", "df64", "c64"):
        h, st, _ = _run_timed(ok, circuit, torch, stream, n, dt, 5, 8, True, ops, [], psi)
        dense[dt] = (ok.orkan_to_dense(h), st)
        ok.orkan_free(h)
    row = {}
    for dt in ("df64", "c64"):
        a, b = dense[dt][0], dense["c128"][0]
        row[dt] = {"max_abs": D.max_abs_diff(a, b), "frobenius": D.frobenius_diff(a, b),
                   "trace_distance": D.trace_distance(a, b), "trace_error": dense[dt][1]["trace_error"]}
    row["c128_trace_error"] = dense["c128"][1]["trace_error"]
    out["n12_vs_gpu_c128"] = row
    del dense
    # n = 16 (c128 reference) and n = 17 (df64 reference): sampled elements
    for n, refdt, dts in ((16, "c128", ("df64", "c64")), (17, "df64", ("c64",))):
        psi, ops = states(n, None)
        rng = S.rng_for(99 + n)
        N = 1 << n
        rows_i = rng.integers(0, N, 1 << 20)
        cols_i = rng.integers(0, N, 1 << 20)
        diag_i = rng.integers(0, N, 1 << 16)
        rows_i = np.concatenate([rows_i, diag_i])
        cols_i = np.concatenate([cols_i, diag_i])
        h, st_ref, _ = _run_timed(ok, circuit, torch, stream, n, refdt, 5, 8, True, ops, [], psi)
        ref_s = ok.orkan_get_elements(h, rows_i, cols_i)
        ok.orkan_free(h)
        row = {"reference": refdt, "reference_ops_per_s": st_ref["ops_per_s"], "sampled_elements": int(rows_i.size),
               "reference_trace_error": st_ref["trace_error"]}
        for dt in dts:
            h, st, _ = _run_timed(ok, circuit, torch, stream, n, dt, 5, 8, True, ops, [], psi)
            got = ok.orkan_get_elements(h, rows_i, cols_i)
            ok.orkan_free(h)
            d = got - ref_s
            row[dt] = {"max_abs_sampled": float(np.max(np.abs(d))),
                       "frobenius_estimate": float(np.sqrt(np.mean(np.abs(d) ** 2)) * N),
                       "trace_distance_bound": float(np.sqrt(np.mean(np.abs(d) ** 2)) * N * np.sqrt(N)),
                       "trace_error": st["trace_error"], "ops_per_s": st["ops_per_s"]}
        out[f"n{n}_vs_gpu_{refdt}"] = row
    return out


def time_steps(runner, steps, warmup, torch):
    for _ in range(warmup):
        runner.step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    l0 = runner.launches()
    runner.timing(True)
    runner.pass_time()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(steps):
        runner.step()
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    pass_ms, pass_cnt = runner.pass_time()
    runner.timing(False)
    return ms, pass_ms, pass_cnt, runner.launches() - l0


def _sample_ops(wl):
    """The CPU sample: the sweep's single-qubit Haar unitaries (the cheapest
    op class for the dense oracle, two N x N products each)."""
    return [op for op in wl["ops"] if op["kind"] == "unitary" and len(op["qubits"]) == 1]


def cpu_baseline(wl, n, seconds):
    """The oracle as it stands, on the same sweep at the same n, until the time
    budget is spent (at least one op); returns ops/s and the sample."""
    import numpy as np
    from oracle import dense as D
    psi = wl["psi"]
    rho = np.outer(psi, psi.conj())
    t0 = time.perf_counter()
    done = 0
    for op in _sample_ops(wl):
        rho, _ = D.apply_op(rho, op)
        done += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} single-qubit Haar unitaries of the n={n} sweep on a dense complex128 rho "
                      f"(scipy.sparse Kronecker K, single-threaded), {dt:.1f} s"}


def run_reference(args):
    """--impl reference: the oracle, timed as it stands on the host cores,
    one single-qubit unitary of the n-qubit sweep per step."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    from oracle import dense as D
    wl = make_workload(args.n)
    ops = _sample_ops(wl)
    psi = wl["psi"]
    rho = np.outer(psi, psi.conj())
    k = 0
    for _ in range(args.warmup):
        rho, _ = D.apply_op(rho, ops[k % len(ops)])
        k += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rho, _ = D.apply_op(rho, ops[k % len(ops)])
        k += 1
    dt = time.perf_counter() - t0
    v = args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": f"per-op sweep n={args.n}: one single-qubit Haar unitary of the sweep per step "
                               f"(dense complex128 oracle)", "n": args.n},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} single-qubit Haar unitaries of the n={args.n} sweep, one per step"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    bound_cores = bind_near_gpu(torch, torch.cuda.current_device())
    from paper_2604_15765_gb300 import build as _b
    _b.build()
    from paper_2604_15765_gb300 import circuit
    from paper_2604_15765_gb300 import orkan as ok

    n, m = args.n, args.tile_log2
    wl = make_workload(n)
    stream = torch.cuda.current_stream().cuda_stream
    if args.op_class:
        tab = per_op_table(ok, wl, n, m, (args.dtype,), stream, torch, reps=args.steps, only=args.op_class)
        print(json.dumps({"op_class": args.op_class, "dtype": args.dtype, "n": n, "pass_GBps": tab[args.dtype]}))
        return 0
    if args.workload == "pipes":
        # the measured pipe rates behind the derived ALU peaks (per SM per clock at the sampled SM clock)
        scratch = torch.empty(4 << 30, dtype=torch.uint8, device="cuda")
        with ClockSampler(gpu_uuid(torch, local)) as cs:
            rates = ok.orkan_probe_pipes(scratch.data_ptr(), scratch.numel())
        clocks = cs.summary()
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        mhz = clocks.get("sm_mhz") or 2070.0
        per = {k.replace("_per_s", "_per_sm_clk"): round(v / sms / (mhz * 1e6), 2) for k, v in rates.items() if k.endswith("_per_s")}
        print(json.dumps({"workload": "pipes", "sms": sms, "rates": rates, "per_sm_per_clock": per, "clocks": clocks,
                          "derived_alu_peaks_T": {k: alu_peak_tops(k, sms) for k in UNIT_RATE}}), flush=True)
        return 0
    if args.workload in ("brickwork", "precision", "paper", "relabel"):
        if args.workload == "relabel":
            rl = relabel_study(ok, circuit, torch, stream, n=16 if args.n == 14 else args.n, depth=args.depth)
            val = rl[args.dtype]["relabel"]["ops_per_s"] if args.dtype in rl else rl["df64"]["relabel"]["ops_per_s"]
            cfg = {"workload": f"circuit on the 5 highest of n={rl['n']} qubits, depth {args.depth}: automatic "
                               "qubit relabelling vs none", "n": rl["n"], "depth": args.depth}
            extra = {"relabel": rl}
        elif args.workload == "paper":
            ps = paper_study(ok, torch, stream, dtypes=tuple(args.paper_dtypes.split(",")),
                             ns=tuple(int(x) for x in args.paper_sizes.split(",")),
                             experiments=tuple(args.paper_ops.split(",")), layouts=tuple(args.paper_layouts.split(",")))
            full = "16" in ps.get("df64", {}) and all(k in ps["df64"]["16"] for k in ("depolarize", "x", "hadamard", "cnot"))
            big = ps["df64"]["16"] if full else None
            ops = 3 * 16 + 16 * 15   # depolarising, X and Hadamard on 16 targets, CNOT on 240 ordered pairs
            if big is not None and all("tiled_fused_us" in big[k] for k in ("depolarize", "x", "hadamard", "cnot")):
                secs = sum(big[k]["tiled_fused_us"] * (16 * 15 if k == "cnot" else 16) for k in
                           ("depolarize", "x", "hadamard", "cnot")) * 1e-6
                val = round(ops / secs, 2)
            else:
                val = None   # a partial study (selected sizes / experiments) has no headline value
            cfg = {"workload": "the paper's experiments: depolarising p=0.1, X, Hadamard, CNOT over all positions, "
                               "n=6..16, packed column-major vs tiled (m=5) one op per pass vs tiled fused; value = "
                               "tiled fused ops/s over the four experiments at n=16 in df64"}
            extra = {"paper": ps}
        elif args.workload == "brickwork":
            bw = brickwork_study(ok, circuit, torch, stream, 16 if args.n == 14 else args.n, args.dtype, args.depth)
            val = bw["autotuned"]["ops_per_s"]
            cfg = {"workload": f"noisy brickwork n={bw['n']}, depth {args.depth}, autotuned vs unfused",
                   "n": bw["n"], "depth": args.depth}
            extra = {"brickwork": bw}
        else:
            pr = precision_study(ok, circuit, torch, stream, args.depth)
            val = pr["n16_vs_gpu_c128"]["df64"]["ops_per_s"]
            cfg = {"workload": f"precision study: noisy brickwork depth {args.depth} at n=10/12/16/17"}
            extra = {"precision": pr}
        line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": 1, "warmup": 0,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
                "data": "synthetic", "config": cfg}
        line.update(extra)
        print(json.dumps(line), flush=True)
        return 0
    if args.workload == "tensor":
        # complex64 in-tile runs: CUDA-core fused pass vs the tensor-core pass of the composed block
        ts = tensor_study(ok, circuit, args.n, m, stream, reps=args.steps)
        print(json.dumps({"workload": "tensor", "metric": "in-tile run time and pass GB/s", "tensor_core_c64": ts}),
              flush=True)
        return 0
    if args.workload == "batch":
        # the batched persistent launch on 300 served requests of n = 4..8 at one dtype, one launch
        from paper_2604_15765_gb300 import serving
        from workloads import synth as S
        dt = args.dtype if args.dtype in ("c128", "c64") else "c128"
        reqs = serving.prepare([dict(r, dtype=dt) for r in
                                S.serving_stream(count=300, seed=S.BASE_SEED + 16, n_range=(4, 8))])
        pool = serving.HandlePool(8 << 30)
        serving.run_batched(pool, reqs[:8])
        torch.cuda.synchronize()
        times = []
        for _ in range(max(args.steps, 1) + 1):   # the first call also allocates the pool's handles
            t0 = time.perf_counter()
            serving.run_batched(pool, reqs)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        pool.close()
        first, dt_s = times[0], statistics.median(times[1:])
        print(json.dumps({"workload": "batch", "dtype": dt, "requests": len(reqs), "solves_per_s": len(reqs) / dt_s,
                          "ops_per_s": sum(len(r["ops"]) for r in reqs) / dt_s, "timed_calls": len(times) - 1,
                          "first_call_solves_per_s": len(reqs) / first}), flush=True)
        return 0
    if args.workload == "serving":
        from workloads import synth as S
        reqs = S.serving_stream(count=5000)
        from paper_2604_15765_gb300 import serving as _sv
        _sv.prepare(reqs)
        if world > 1:
            # request-level replicas: each rank serves its routed share on its own GPU, nothing is
            # exchanged while requests run; results and latencies are gathered once at the end
            from paper_2604_15765_gb300 import serving
            _, cap = serving.serve_replicated(reqs, 64 << 30, slots=8, realtime=False, batch_max_n=8)
            st = {"replicated_capacity": cap}
        else:
            st = serving_study(reqs, torch, budget=64 << 30, realtime_fracs=(0.5, 0.9, 1.2))
            cap = st["served_capacity"]
        if rank != 0:
            return 0
        line = {"metric": METRIC, "value": round(cap["ops_per_s"], 2), "unit": UNIT, "n_gpus": world, "steps": 1,
                "warmup": 0, "ms_per_step": round(cap["elapsed_s"] * 1e3, 1), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "c128/c64 requests, each at its own dtype",
                "data": "synthetic",
                "config": {"workload": "serving: 5000 seeded requests, n~U{4..14}, depth~U{10..200} from the "
                                       "mixed op mix, 50/50 picture and dtype"},
                "serving": st}
        print(json.dumps(line), flush=True)
        return 0
    compose = not args.no_compose
    runner = Runner(ok, circuit, wl, n, m, args.dtype, args.fusion, compose, stream)

    # ---- device-resident throughput
    gpu_id = gpu_uuid(torch, local)
    with ClockSampler(gpu_id) as clk:
        ms, pass_ms, pass_cnt, launches = time_steps(runner, args.steps, args.warmup, torch)
    clocks = clk.summary()
    units = runner.ops_per_step * args.steps
    tot_units, tot_s = aggregate(units, ms / 1e3)
    value = tot_units / tot_s

    # ---- end to end through the C ABI from pinned host buffers
    host_rho = torch.empty(runner.bytes, dtype=torch.uint8, pin_memory=True)
    host_O = torch.empty(runner.bytes, dtype=torch.uint8, pin_memory=True)
    ok.orkan_store_tiled(runner.rho, host_rho.numpy())
    ok.orkan_store_tiled(runner.O, host_O.numpy())
    e2e_steps = max(2, args.steps // 2)
    # Two handle pairs alternate, as a server double-buffers requests: before
    # step i runs on one pair, the uploads of step i + 1's inputs are queued on
    # the other pair's streams, so they overlap step i's passes; every step's
    # copies (the first one included) are inside the timed region.  Within a
    # pair the observable has a stream of its own: its passes follow its copy
    # there, and tr(rho O) waits for that stream.  A step ends with blocking
    # readouts, so the pair it used is idle when its next upload is queued.
    # Copy durations are timed with events on the copies' own streams.
    s_rho = torch.cuda.current_stream()   # the first pair's state stream (the runner's `stream`)
    s_rho2, stream_o, stream_o2 = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    runner2 = Runner(ok, circuit, wl, n, m, args.dtype, args.fusion, compose, s_rho2.cuda_stream)
    ok.orkan_set_stream(runner.O, stream_o.cuda_stream)
    ok.orkan_set_stream(runner2.O, stream_o2.cuda_stream)
    pairs = [(runner, s_rho, stream_o), (runner2, s_rho2, stream_o2)]
    copy_ev = []

    def upload(k):
        r, sr, so = pairs[k]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(sr)
        ok.orkan_load_tiled_async(r.rho, host_rho.numpy(), ok.ORKAN_STATE)
        ev[1].record(sr)
        ev[2].record(so)
        ok.orkan_load_tiled_async(r.O, host_O.numpy(), ok.ORKAN_OBSERVABLE)
        ev[3].record(so)
        copy_ev.append(ev)

    def e2e_steps_run(count):
        upload(0)
        for i in range(count):
            if i + 1 < count:
                upload((i + 1) % 2)
            pairs[i % 2][0].step()                                          # ends with blocking readouts

    e2e_steps_run(2)                                                        # warms both pairs
    torch.cuda.synchronize()
    barrier()
    copy_ev.clear()
    t0 = time.perf_counter()
    e2e_steps_run(e2e_steps)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    upload_ms = sum(ev[0].elapsed_time(ev[1]) + ev[2].elapsed_time(ev[3]) for ev in copy_ev) / e2e_steps
    ok.orkan_set_stream(runner.O, stream)
    runner2.free()
    e2e_units, e2e_tot = aggregate(runner.ops_per_step * e2e_steps, e2e_s)
    op_bytes = sum(16 * op["matrix"].size if op["kind"] == "unitary" else 8 for op in wl["ops"]) * 2
    h2d = 2 * runner.bytes + op_bytes
    d2h = 8 * (1 + len(wl["paulis"]) + 2 + 1) + 8

    # ---- roofline of the dominant kernel (the fused pass kernel), on the HBM basis: algorithmic bytes
    # (2 x stored bytes per pass) / average pass duration / measured copy bandwidth.  The pipe that
    # does the arithmetic (FP64 for c128) is reported beside it as its own field.
    hbm_peak, peak_kind = peaks()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    avg_pass_ms = pass_ms / max(pass_cnt, 1)
    achieved = 2.0 * runner.bytes / (avg_pass_ms * 1e-3) / 1e9
    alu_ops = runner.work[0]
    alu_tops = alu_ops / (pass_ms * 1e-3) / 1e12 if pass_ms > 0 else 0.0
    alu_peak = alu_peak_tops(args.dtype, sms)
    trec = traffic_record(args.dtype)
    pipe_name = "fp64_pipe" if args.dtype == "c128" else "fp32_pipe"
    pipe = {"achieved": round(alu_tops, 4), "peak": round(alu_peak, 4),
            "unit": "Tops/s (" + ("FP64 operations" if args.dtype == "c128" else "FP32 lane operations") + ")",
            "frac": round(alu_tops / alu_peak, 4),
            "peak_kind": f"derived: {sms} SMs (device) x {UNIT_RATE[args.dtype]:g} per SM per clock x 2.07 GHz",
            "algorithmic_ops_per_launch": round(alu_ops / max(pass_cnt, 1)),
            "ops_counted": "the arithmetic each op form needs per stored element (no addressing or data movement)"}
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(achieved / hbm_peak, 4), "traffic": (trec or {}).get("bytes_per_launch"),
                "kernel": "pass_kernel (fused tile-group conjugation)", "peak_kind": f"{peak_kind} hbm_gbs (burst copy)",
                pipe_name: pipe,
                "algorithmic_bytes_per_launch": 2 * runner.bytes, "avg_launch_ms": round(avg_pass_ms, 4),
                "launches": pass_cnt, "pass_share_of_step": round(pass_ms / ms, 4) if ms > 0 else None}
    runner.free()

    # ---- comparison runs (rank 0 only): plain FP64 one-op-per-pass, and the declared faster forms (double-float
    # and complex64), each with its error against the native FP64 run on one Schroedinger sweep
    variants = {}
    if not args.no_variants and world == 1:
        ref_elems, samp = sweep_elements(ok, circuit, wl, n, m, "c128", args.fusion, compose, stream)
        for name, dt, fus, comp in (("c128_plain_unfused", "c128", 1, False), ("c128_fused", "c128", args.fusion, True),
                                    ("df64_fused", "df64", args.fusion, True), ("df64_unfused", "df64", 1, False),
                                    ("c64_fused", "c64", args.fusion, True)):
            if dt == args.dtype and fus == args.fusion and comp == compose:
                continue
            r = Runner(ok, circuit, wl, n, m, dt, fus, comp, stream)
            vms, vpass, vcnt, _ = time_steps(r, max(2, args.steps // 3), 1, torch)
            variants[name] = {"value": round(r.ops_per_step * max(2, args.steps // 3) / (vms / 1e3), 1), "unit": UNIT,
                              "dtype": dt, "fusion": fus,
                              "avg_pass_GBps": round(2.0 * r.bytes / (vpass / max(vcnt, 1) * 1e-3) / 1e9, 1)}
            r.free()
            got, _ = sweep_elements(ok, circuit, wl, n, m, dt, fus, comp, stream, samp)
            variants[name]["max_abs_err_vs_c128"] = float(np.max(np.abs(got - ref_elems)))
            variants[name]["error_sample"] = (f"{samp[0].size} sampled elements (incl. {samp[2]} diagonal) after one "
                                              f"Schroedinger sweep, against the native FP64 fused run")

    bw16 = None
    if not args.no_variants and world == 1 and args.bw_depth > 0:
        bw16 = brickwork_prefix(ok, circuit, torch, stream, 16, "c128", args.bw_depth, hbm_peak)

    per_op = None
    serving_res = None
    if not args.no_variants and world == 1:
        per_op = per_op_table(ok, wl, n, m, ("df64", "c128", "c64"), stream, torch)
        per_op["tensor_core_c64"] = tensor_study(ok, circuit, n, m, stream)
        from workloads import synth as S
        serving_res = serving_study(S.serving_stream(count=args.serve_requests), torch, budget=32 << 30)
        serving_res["small_requests"] = small_request_study(S, torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, n, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(tot_s * 1e3 / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": f"per-op sweep n={n}, tiled m={m}: every target, 1q Haar U + depolarising p=0.1 "
                                   f"+ amplitude damping 0.05 + 2q Haar U adjacent and far; Schroedinger + "
                                   f"Heisenberg; Z measurement, 8 Pauli expectations, trace, tr(rho O)",
                       "n": n, "tile_log2": m, "fusion": args.fusion, "compose": compose,
                       "ops_per_step": runner.ops_per_step, "state_bytes": runner.bytes,
                       "l2": "no flush: each operand (%.2f GB) is larger than the 129 MB L2" % (runner.bytes / 1e9),
                       "parallelism": f"replicas{world}"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_units / e2e_tot, 2), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "host_cores_near_gpu": bound_cores,
                    "upload_ms_per_step": round(upload_ms, 2),
                    "ms_per_step": round(1e3 * e2e_s / e2e_steps, 2),
                    "uploads": "asynchronous from pinned memory into two alternating handle pairs: each step's "
                               "copies overlap the previous step's passes"},
            "gpu_launches": launches,
            "clocks": clocks,
            "variants": variants,
            "brickwork_n16": bw16,
            "per_op_pass_GBps": per_op,
            "serving": serving_res,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
