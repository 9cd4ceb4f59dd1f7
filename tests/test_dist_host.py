"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

Problems are independent replicas, so the only cross-rank operations are the timing
reduction (max over ranks) and the unit count (sum over ranks); the reference arm runs on
rank 0 only.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    d = bench.init_dist(w, "gloo")
    bench.barrier(d)
    secs, units = bench.aggregate(d, 1.0 + rank, 100.0 * (rank + 1))
    # the reference arm is rank 0's job; other ranks exit 0 without work
    ref_rc = None
    if rank != 0:
        ref_rc = bench.run_reference(type("A", (), {"workload": "small", "warmup": 3, "steps": 1})())
    out.put((rank, secs, units, ref_rc))
    dist.destroy_process_group()


def test_aggregate_and_rank0_only_reference_on_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, secs, units, ref_rc in res:
        assert secs == 2.0            # max over ranks
        assert units == 300.0         # sum over ranks
        if rank == 1:
            assert ref_rc == 0


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.init_dist(1, "gloo") is None
    assert bench.aggregate(None, 3.0, 7.0) == (3.0, 7.0)
