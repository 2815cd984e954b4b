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
