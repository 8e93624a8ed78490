"""The multi-process path of bench.py on CPU: two gloo ranks combine their
replicas' timings the way the GPU run does (slowest rank's time, sum of the
updates), and the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from tests.conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.combine_ranks(1.5 + rank, 1000 * (rank + 1), "cpu")
    ws, r, local = bench.dist_env()
    out[rank] = (t, u, ws, r, local)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_combination():
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        t, u, ws, rr, local = out[r]
        assert t == 2.5 and u == 3000.0
        assert ws == 2 and rr == r and local == r


def test_reference_arm_other_ranks_exit(monkeypatch, capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class Args:
        steps, warmup, ref_budget_s = 1, 0, 1.0
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""


def test_launch_count_follows_the_step_structure():
    """gpu_launches: after a restore the first step hashes in a pass of its
    own (5 launches: hash, flood, scan, gather, pedestrian update); then 4 per
    step with hash-ahead and no barrier, else 5 -- the per-kernel launch
    counts of the ncu launch list of 64 steps."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import scenarios
    plain = scenarios.config_shopping()
    assert bench.launches_per_chunk(plain, True) == 5 + (bench.CHUNK - 1) * 4
    assert bench.launches_per_chunk(plain, False) == 5 * bench.CHUNK
    barrier = scenarios.shopping_centre(128, 0.5, 100, 10, 1, 600.0, n_barrier=8, n_layers=2)
    assert bench.launches_per_chunk(barrier, True) == 5 * bench.CHUNK
