"""The benchmark's multi-rank path on CPU: two gloo ranks (world size 2).

Under torchrun each rank draws its own population and times its own steps;
the job's time is the slowest rank's and its throughput counts the units of
every rank.  The same helpers run here with gloo and CPU tensors."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2108_10565_gb300 import inputs
        t = bench.max_over_ranks(0.5 + 0.25 * rank, world, "cpu")  # rank 1 is the slower one
        pop = inputs.isolated_elements(8, 2, seed=bench.rank_seed(rank))
        res = {"t": t, "rate": bench.job_rate(1000, world, t), "seed": bench.rank_seed(rank),
               "q0_sum": float(pop["Q0"].sum())}
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump(res, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(world)]
    # the slowest rank's time on every rank, and the job rate counts both ranks
    assert r[0]["t"] == r[1]["t"] == 0.75
    assert r[0]["rate"] == r[1]["rate"] == pytest.approx(1000 * 2 / 0.75)
    # each rank has its own population (no shared data, weak scaling)
    assert r[0]["seed"] != r[1]["seed"] and r[0]["q0_sum"] != r[1]["q0_sum"]


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.3, 1, "cpu") == 0.3
    assert bench.job_rate(200_000, 1, 0.0814) == pytest.approx(200_000 / 0.0814)
