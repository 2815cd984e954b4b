"""Multi-rank host logic on CPU (gloo, world size 2): every rank runs an
independent replica; the job's throughput is the sum of the ranks' ops over
the slowest rank's time, and the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units, secs = bench.aggregate(100.0 * (rank + 1), 1.5 + rank)
    bench.barrier()
    # the reference arm: ranks other than 0 return without work or output
    rc = bench.run_reference(bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "0", "--n", "3"])) \
        if rank == 1 else 0
    q.put((rank, units, secs, rc))
    dist.destroy_process_group()


def test_aggregate_sum_over_max_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, units, secs, rc in res:
        assert units == pytest.approx(300.0)
        assert secs == pytest.approx(2.5)
        assert rc == 0


def test_cpulist_parsing():
    import bench
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("5") == {5}
    assert bench.parse_cpulist("") == set()


def _fake_serve(reqs, budget, **kw):
    """Host-only stand-in for one replica's serve(): result = the request id."""
    import numpy as np
    import torch.distributed as dist
    rank = dist.get_rank() if dist.is_initialized() else 0
    res = {r["id"]: np.array([float(r["id"])]) for r in reqs}
    return res, {"requests": len(reqs), "elapsed_s": 1.0 + rank, "ops_per_s": 10.0 * len(reqs) / (1.0 + rank),
                 "latencies_s": [0.001 * (1 + rank)] * len(reqs)}


def _route_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2604_15765_gb300 import serving
    from workloads import synth as S
    reqs = S.serving_stream(count=40, n_range=(4, 9), depth_range=(5, 30))
    mine = serving.route(reqs, world)[rank]
    res, st = serving.serve_replicated(reqs, 1 << 30, serve_fn=_fake_serve)
    q.put((rank, sorted(r["id"] for r in mine), sorted(res), st))
    dist.destroy_process_group()


def test_request_level_replicas_gloo():
    """World size 2: the routing gives every request to exactly one rank, no
    data-path exchange is needed (each rank computes the same assignment),
    and the gathered result holds every request once with solves/s = all
    requests / the slowest replica's time.  Unmeasured on GPU hardware: each
    box has one GPU."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_route_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, ids0, got0, st0), (_, ids1, got1, st1) = out
    assert ids0 and ids1 and not set(ids0) & set(ids1)
    assert sorted(ids0 + ids1) == list(range(40))
    assert got0 == got1 == list(range(40))
    for st in (st0, st1):
        assert st["requests"] == 40 and st["replicas"] == 2
        assert st["elapsed_s"] == pytest.approx(2.0)
        assert st["solves_per_s"] == pytest.approx(20.0)


def test_route_balances_estimated_work():
    from paper_2604_15765_gb300 import serving
    from workloads import synth as S
    reqs = S.serving_stream(count=200, n_range=(4, 12))
    for world in (1, 2, 3, 8):
        parts = serving.route(reqs, world)
        assert sorted(r["id"] for p in parts for r in p) == list(range(200))
        assert parts == serving.route(reqs, world)            # deterministic
        loads = [sum(serving.request_cost(r) for r in p) for p in parts]
        biggest = max(serving.request_cost(r) for r in reqs)
        assert max(loads) - min(loads) <= biggest
        for p in parts:
            assert [r["t"] for r in p] == sorted(r["t"] for r in p)
