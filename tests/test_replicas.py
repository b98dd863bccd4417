"""Multi-GPU path of bench.py (replicas only: every rank its own independent
patterns, no data exchange; the max time over ranks; rank 0 reports), run as
two gloo ranks on the CPU."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    import bench
    w = bench.replica_workload("config4_batched", 8, rank, world)
    d = torch.tensor(np.asarray(w.drive_delay), dtype=torch.float64)
    got = [torch.zeros_like(d) for _ in range(world)]
    dist.all_gather(got, d)
    again = bench.replica_workload("config4_batched", 8, rank, world)
    t = bench.max_over_ranks(1.5 + rank, dist, device="cpu")
    out[rank] = dict(
        differ=not torch.equal(got[0], got[1]),
        mine=torch.equal(got[rank], d),
        deterministic=bool(np.array_equal(again.drive_delay, w.drive_delay)),
        tmax=t,
        rate=bench.whole_job_rate(1000, 8, 10, world, t),
    )
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_two_gloo_ranks():
    import torch.multiprocessing as mp
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r]["differ"] and res[r]["mine"] and res[r]["deterministic"]
        assert res[r]["tmax"] == 2.5                     # max over ranks, seen by every rank
        assert res[r]["rate"] == pytest.approx(1000 * 8 * 10 * world / 2.5 / 1e9)


def test_single_rank_workload_is_the_bench_default():
    import bench
    w1 = bench.replica_workload("config4_batched", 8, 0, 1)
    w2 = bench.make_workload("config4_batched", 8)
    assert np.array_equal(w1.drive_delay, w2.drive_delay)
    assert bench.max_over_ranks(3.25, None) == 3.25


def test_reference_arm_other_ranks_exit_without_work(capsys, monkeypatch):
    """Under torchrun only rank 0 runs the reference arm; the others return
    at once and print nothing."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(bench.parse([]))
    assert capsys.readouterr().out == ""
