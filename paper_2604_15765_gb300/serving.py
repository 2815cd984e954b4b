"""Request serving over the Orkan C ABI: continuous batching of mixed-size simulations.

A request (from ``workloads.synth.serving_stream``) is one circuit on one
operator:
  * Schroedinger: start from a product state rho0, apply the circuit (unitaries,
    channels, Z measurements with the request's draws), return 8 Pauli-string
    expectations;
  * Heisenberg: start from a 16-term Pauli-sum observable O, apply the adjoint
    circuit in reverse order, return tr(O rho0) for the request's product
    state rho0.

The server keeps every operator resident in HBM (handles are pooled per
(n, dtype) and reused), admits a request once it has arrived and its packed
tile bytes fit the memory budget, and runs admitted requests concurrently:
each of ``slots`` worker threads owns its own handles and therefore its own
CUDA streams, so the passes of different requests overlap on the GPU while
new requests are admitted as slots and memory free up.  The Python layer only
issues C-ABI calls (ctypes releases the interpreter lock during each call);
every step of every circuit runs in the library's kernels.

Results are deterministic per request: each kernel's grid and reduction order
depend only on the request's own operator, never on what else is running.
"""
from __future__ import annotations

import collections
import heapq
import threading
import time

import numpy as np

from . import circuit
from . import orkan as ok

DT = {"c128": ok.ORKAN_C128, "c64": ok.ORKAN_C64, "df64": ok.ORKAN_DF64}


class HandlePool:
    """Resident operators per (n, dtype, tile_log2), with memory accounting."""

    def __init__(self, budget_bytes: int, tile_log2: int = 5):
        self.budget = int(budget_bytes)
        self.m = tile_log2
        self.free = collections.defaultdict(list)
        self.allocated = 0
        self.lock = threading.Lock()
        self.cv = threading.Condition(self.lock)

    def nbytes(self, n, dtype):
        return ok.orkan_bytes(n, DT[dtype], self.m)

    def _evict_idle(self, need):
        for key in list(self.free):
            while self.free[key] and self.allocated + need > self.budget:
                h = self.free[key].pop()
                ok.orkan_free(h)
                self.allocated -= self.nbytes(key[0], key[1])

    def acquire(self, n, dtype, count=1, block=True):
        """count handles for an n-qubit operator, or None if not admissible now.
        A request that could never fit the budget raises ValueError instead of
        waiting for memory that will not come."""
        need_each = self.nbytes(n, dtype)
        if need_each * count > self.budget:
            raise ValueError(f"{count} operator(s) of n = {n} ({dtype}, {need_each} bytes each) exceed the "
                             f"memory budget of {self.budget} bytes")
        with self.cv:
            while True:
                reuse = min(count, len(self.free[(n, dtype)]))
                need = need_each * (count - reuse)
                if self.allocated + need > self.budget:
                    self._evict_idle(need)
                if self.allocated + need <= self.budget:
                    hs = [self.free[(n, dtype)].pop() for _ in range(reuse)]
                    for _ in range(count - reuse):
                        hs.append(ok.orkan_alloc(n, DT[dtype], self.m))
                        self.allocated += need_each
                    return hs
                if not block:
                    return None
                self.cv.wait(timeout=0.05)

    def release(self, n, dtype, hs):
        with self.cv:
            self.free[(n, dtype)].extend(hs)
            self.cv.notify_all()

    def close(self):
        with self.cv:
            for key, hs in self.free.items():
                for h in hs:
                    ok.orkan_free(h)
            self.free.clear()
            self.allocated = 0


def run_request(pool: HandlePool, req, dtype_map=None, fusion=8, compose=True):
    """Execute one request on pooled handles; returns its result vector."""
    dtype = (dtype_map or {}).get(req["dtype"], req["dtype"])
    n = req["n"]
    if req["picture"] == "schrodinger":
        (h,) = pool.acquire(n, dtype, 1)
        try:
            ok.orkan_set_fusion(h, fusion, compose)
            ok.orkan_init_state(h, ok.ORKAN_INIT_PURE, req["psi0"])
            circuit.run_circuit(h, req["ops"], "schrodinger", marshalled=marshalled(req))
            out = np.array([ok.orkan_expect_pauli(h, s) for s in req["paulis"]])
        finally:
            pool.release(n, dtype, [h])
        return out
    hO, h0 = pool.acquire(n, dtype, 2)
    try:
        ok.orkan_set_fusion(hO, fusion, compose)
        ok.orkan_init_observable(hO, req["paulis"], req["coeffs"])
        circuit.run_circuit(hO, list(reversed(req["ops"])), "heisenberg", marshalled=marshalled(req))
        ok.orkan_init_state(h0, ok.ORKAN_INIT_PURE, req["psi0"])
        out = np.array([ok.orkan_expect(h0, hO)])
    finally:
        pool.release(n, dtype, [hO, h0])
    return out


def marshalled(req):
    """The request's circuit as a C-ABI op array, made once and kept with the
    request (the form a client hands the server): the ops in order for
    Schroedinger requests, in reverse order for Heisenberg ones."""
    m = req.get("_marshalled")
    if m is None:
        ops = req["ops"] if req["picture"] == "schrodinger" else list(reversed(req["ops"]))
        m = circuit.marshal(ops, req["picture"])
        req["_marshalled"] = m
    return m


def prepare(requests):
    """Marshal every request's circuit up front (see ``marshalled``)."""
    for r in requests:
        marshalled(r)
    return requests


def batch_item(pool: HandlePool, req, dtype_map=None):
    """One request as an orkan_run_batch item on a pooled handle (the whole
    circuit and its readouts in the batched launch): Schroedinger from the
    product state psi0, returning the Pauli expectations; Heisenberg from the
    Pauli sum, the adjoint circuit in reverse order, returning
    <psi0|O|psi0> = tr(O rho0)."""
    dtype = (dtype_map or {}).get(req["dtype"], req["dtype"])
    (h,) = pool.acquire(req["n"], dtype, 1)
    if req["picture"] == "schrodinger":
        item = {"h": h, "init": "pure", "psi0": req["psi0"], "ops": req["ops"], "paulis": req["paulis"],
                "marshalled": marshalled(req)}
    else:
        item = {"h": h, "init": "pauli_sum", "terms": req["paulis"], "coeffs": req["coeffs"],
                "ops": list(reversed(req["ops"])), "psi": req["psi0"], "marshalled": marshalled(req)}
    return item, (req["n"], dtype, h)


def run_batched(pool: HandlePool, reqs, dtype_map=None):
    """Run requests in one orkan_run_batch call; returns their result vectors."""
    # longest estimated work first: the queue hands them out first, which
    # shortens the launch's makespan
    order = sorted(range(len(reqs)), key=lambda i: (-request_cost(reqs[i]), i))
    items, held = [], []
    try:
        for i in order:
            it, hd = batch_item(pool, reqs[i], dtype_map)
            items.append(it)
            held.append(hd)
        out = circuit.run_batch(items)
    finally:
        for n, dt, h in held:
            pool.release(n, dt, [h])
    res = [None] * len(reqs)
    for i, x in zip(order, out):
        res[i] = x
    for r, x in zip(reqs, res):
        if x["status"] != ok.ORKAN_OK:
            raise ok.OrkanError(x["status"], "serve", f"request {r['id']} failed in the batched launch")
    return [x["out"] for x in res]


def request_cost(req) -> float:
    """Estimated device work of a request: ops x stored elements (~4^n)."""
    return float(len(req["ops"])) * 4.0 ** req["n"]


def serve(requests, budget_bytes, slots=8, dtype_map=None, fusion=8, compose=True, realtime=True,
          tile_log2=5, policy="fifo", batch_max_n=None, batch_size=256, latencies=False):
    """Continuous batching: requests become eligible at their arrival time
    (offsets from the start when ``realtime``), are admitted when a slot is
    free and their bytes fit the budget, and run concurrently.  ``policy``
    orders the eligible requests: "fifo" by arrival, "sjf" shortest estimated
    work first (``request_cost``; ties by arrival).  With ``batch_max_n``,
    requests of at most that many qubits do not take a slot: one more worker
    collects every eligible one (up to ``batch_size``, within half the memory
    budget) into a single orkan_run_batch launch, again and again, while
    larger requests run on the slots.  Returns (results by request id,
    stats); with ``latencies`` the stats also list every request's latency.
    One replica on one GPU; ``serve_replicated`` spreads requests over
    torch.distributed ranks."""
    if policy not in ("fifo", "sjf"):
        raise ValueError(policy)
    pool = HandlePool(budget_bytes, tile_log2)
    order = sorted(requests, key=lambda r: r["t"])
    arrived = [0]          # requests of `order` moved to an eligible heap so far
    eligible = [[], []]    # (key, seq, request): [0] slot requests, [1] batched requests
    qlock = threading.Lock()
    results, lat = {}, {}
    errors = []
    t0 = time.perf_counter()

    def small(r):
        return batch_max_n is not None and r["n"] <= batch_max_n

    def admit(now):
        while arrived[0] < len(order) and (not realtime or order[arrived[0]]["t"] <= now):
            r = order[arrived[0]]
            key = request_cost(r) if policy == "sjf" else r["t"]
            heapq.heappush(eligible[1 if small(r) else 0], (key, arrived[0], r))
            arrived[0] += 1

    def take(which, count):
        """Up to `count` eligible requests of one kind ([] when none will come)."""
        while True:
            with qlock:
                now = time.perf_counter() - t0
                admit(now)
                if eligible[which]:
                    out, mem = [], 0
                    while eligible[which] and len(out) < count:
                        r = eligible[which][0][2]
                        need = pool.nbytes(r["n"], (dtype_map or {}).get(r["dtype"], r["dtype"]))
                        if out and mem + need > budget_bytes // 2:
                            break
                        heapq.heappop(eligible[which])
                        out.append(r)
                        mem += need
                    return out
                if arrived[0] >= len(order):
                    return []
                wait = order[arrived[0]]["t"] - now
            time.sleep(max(wait, 0.0))

    def done(req, res):
        t = time.perf_counter()
        results[req["id"]] = res
        lat[req["id"]] = t - (t0 + req["t"] if realtime else t0)

    def worker():
        while True:
            got = take(0, 1)
            if not got:
                return
            req = got[0]
            try:
                res = run_request(pool, req, dtype_map, fusion, compose)
            except Exception as e:  # noqa: BLE001  (reported to the caller)
                errors.append((req["id"], repr(e)))
                continue
            done(req, res)

    def batch_worker():
        while True:
            got = take(1, batch_size)
            if not got:
                return
            try:
                res = run_batched(pool, got, dtype_map)
            except Exception as e:  # noqa: BLE001
                errors.append((got[0]["id"], repr(e)))
                continue
            for r, x in zip(got, res):
                done(r, x)

    threads = [threading.Thread(target=worker, daemon=True) for _ in range(slots)]
    if batch_max_n is not None:
        threads.append(threading.Thread(target=batch_worker, daemon=True))
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    elapsed = time.perf_counter() - t0
    pool.close()
    if errors:
        raise RuntimeError(f"{len(errors)} requests failed, first: {errors[0]}")
    lv = np.array(sorted(lat.values())) if lat else np.zeros(1)
    ops = sum(len(r["ops"]) for r in requests)
    stats = {"requests": len(results), "elapsed_s": elapsed, "solves_per_s": len(results) / elapsed,
             "ops_per_s": ops / elapsed, "p50_ms": float(np.percentile(lv, 50) * 1e3),
             "p99_ms": float(np.percentile(lv, 99) * 1e3), "slots": slots, "policy": policy,
             "batch_max_n": batch_max_n}
    if latencies:
        stats["latencies_s"] = [float(x) for x in lv] if lat else []
    return results, stats


# ------------------------------------------------------------------ request-level replicas
def route(requests, world: int):
    """Spread requests over `world` independent replicas (one GPU each): each
    request, in decreasing estimated work (ties by id), goes to the replica
    with the least work so far (ties by rank).  Deterministic, so every rank
    computes the same assignment without communicating.  Returns one request
    list per rank, each in arrival order."""
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for r in sorted(requests, key=lambda r: (-request_cost(r), r["id"])):
        k = min(range(world), key=lambda w: (load[w], w))
        parts[k].append(r)
        load[k] += request_cost(r)
    return [sorted(p, key=lambda r: (r["t"], r["id"])) for p in parts]


def merge_replicas(parts):
    """Combine the (results, stats) of every replica: results by request id;
    solves/s and ops/s = all requests / the slowest replica's elapsed time;
    p50/p99 over every request's latency (each replica reports its own)."""
    results = {}
    lat = []
    elapsed = 0.0
    nreq = 0
    ops = 0.0
    for res, st, lats in parts:
        results.update(res)
        lat.extend(lats)
        elapsed = max(elapsed, st["elapsed_s"])
        nreq += st["requests"]
        ops += st["ops_per_s"] * st["elapsed_s"]
    lv = np.array(sorted(lat)) if lat else np.zeros(1)
    return results, {"requests": nreq, "replicas": len(parts), "elapsed_s": elapsed,
                     "solves_per_s": nreq / elapsed if elapsed > 0 else 0.0,
                     "ops_per_s": ops / elapsed if elapsed > 0 else 0.0,
                     "p50_ms": float(np.percentile(lv, 50) * 1e3), "p99_ms": float(np.percentile(lv, 99) * 1e3)}


def serve_replicated(requests, budget_bytes, group=None, serve_fn=None, **kw):
    """Request-level data parallelism: under torch.distributed every rank
    serves its share (``route``) on its own GPU as an independent replica --
    nothing is exchanged while requests run -- and the ranks gather their
    results and latencies once at the end.  Without an initialised process
    group this is ``serve``.  ``serve_fn`` (default ``serve``) must return
    (results, stats) with stats["latencies_s"]."""
    import torch.distributed as dist
    serve_fn = serve_fn or _serve_with_latencies
    if not (dist.is_available() and dist.is_initialized()):
        res, st = serve_fn(requests, budget_bytes, **kw)
        return merge_replicas([(res, st, st.pop("latencies_s"))])
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    mine = route(requests, world)[rank]
    res, st = serve_fn(mine, budget_bytes, **kw)
    lats = st.pop("latencies_s")
    gathered = [None] * world
    dist.all_gather_object(gathered, (res, st, lats), group=group)
    return merge_replicas(gathered)


def _serve_with_latencies(requests, budget_bytes, **kw):
    if not requests:
        return {}, {"requests": 0, "elapsed_s": 0.0, "ops_per_s": 0.0, "latencies_s": []}
    res, st = serve(requests, budget_bytes, latencies=True, **kw)
    return res, st
