"""Host side of the multi-GPU (replica) path on CPU: world_size-2 gloo process groups.

The residual path does not shard: N GPUs run N independent replicas (one problem per rank, no
collective on the data path), and the only cross-rank step is the timing reduction (barrier +
max over ranks).  These tests run that reduction and the rank handling of bench.py with the gloo
backend on 127.0.0.1.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, ms_local, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_max = bench.max_over_ranks(ms_local[rank], dist, device="cpu")
        value = bench.whole_job_rate(5, world, ms_max)
        p = bench.workload(8, seed=rank)
        q.put((rank, ms_max, value, p.name, float(p.h[0, 1])))
    finally:
        dist.destroy_process_group()


def test_timing_reduction_and_replica_seeds_gloo():
    world, port = 2, _free_port()
    ms_local = [10.0, 20.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, ms_local, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms_max, value, name, h01 in out:
        assert ms_max == 20.0                          # every rank sees the slowest rank's time
        assert value == pytest.approx(2 * 5 / 0.020)   # whole-job rate: all ranks' units / max time
    assert out[0][3] == out[1][3]                      # same workload family on every rank
    assert out[0][4] != out[1][4]                      # independent replicas: rank-seeded inputs


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        r, steps, warmup = 8, 1, 0
    bench.run_reference(Args, rank=1, world=2)
    assert capsys.readouterr().out == ""               # rank 1 exits without work or output
