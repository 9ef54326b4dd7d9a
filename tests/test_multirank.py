"""The multi-rank path of bench.py on CPU: two gloo ranks, one replica each (weak scaling).
The timed totals reduce to the slowest rank's, every rank counts its own units, and the
reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [100.0, 130.0][rank]          # total timed ms of this rank's steps
    e2e = [150.0, 140.0][rank]
    out = bench.aggregate_ranks(torch, ms, e2e, evals=1e9, steps=10, world=world, dist=dist,
                                device="cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def test_two_gloo_ranks_take_the_slowest_rank_and_count_both_replicas():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        ms_per_step, value, e2e_value = res[rank]
        assert ms_per_step == pytest.approx(13.0)            # max over ranks / steps
        assert value == pytest.approx(2 * 1e9 / 13.0e-3)    # both replicas' units
        assert e2e_value == pytest.approx(2 * 1e9 / 15.0e-3)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class Args:
        workload = "open_plane_small"
        steps = 1
        warmup = 0
    assert bench.run_reference(Args()) is None               # returns at once, no work
