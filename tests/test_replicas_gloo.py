"""Replica bookkeeping across two `gloo` ranks on the CPU.

Runs on several GPUs give every rank its own independent requests (weak
scaling, no data-path collective); the only cross-rank steps are the barrier
around the timed region and a MAX of the elapsed times.  These tests run that
logic as two spawned processes with the `gloo` backend.
"""
import os
import socket

import pytest
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

from paper_2607_02630_gb300 import replicas as R
from paper_2607_02630_gb300 import workloads as W


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, elapsed, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    ws, r, local = R.world_from_env()
    tdist.init_process_group("gloo", rank=r, world_size=ws)
    try:
        tdist.barrier()
        worst = R.max_over_ranks(elapsed[rank], tdist, torch.device("cpu"))
        w = W.batch_varlen(n=16, seed=R.rank_seed(W.SEED_BASE + 3, r), with_payload=False)
        step_bytes = int(w.lengths.sum())
        with open(os.path.join(out_dir, f"rank{r}.txt"), "w") as f:
            f.write(f"{ws} {r} {local} {worst!r} {step_bytes} {w.lengths.tolist()}\n")
        tdist.barrier()
    finally:
        tdist.destroy_process_group()


def test_world_from_env_defaults():
    assert R.world_from_env({}) == (1, 0, 0)
    assert R.world_from_env({"WORLD_SIZE": "4", "RANK": "2", "LOCAL_RANK": "1"}) == (4, 2, 1)


def test_max_over_ranks_without_group():
    assert R.max_over_ranks(1.25) == 1.25


def test_aggregate_gbs():
    # 2 ranks x 3 steps x 1e9 bytes over 2 s = 3 GB/s
    assert R.aggregate_gbs(10**9, 3, 2, 2.0) == pytest.approx(3.0)


def test_rank_seeds_distinct():
    seeds = {R.rank_seed(W.SEED_BASE, r) for r in range(8)}
    assert len(seeds) == 8


def test_two_gloo_ranks(tmp_path):
    world = 2
    elapsed = [0.75, 1.5]
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, elapsed, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    for p in procs:
        if p.is_alive():
            p.kill()
            p.join()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    rows = []
    for r in range(world):
        ws, rk, local, worst, step_bytes, lengths = open(tmp_path / f"rank{r}.txt").read().split(" ", 5)
        rows.append((int(ws), int(rk), int(local), float(worst), int(step_bytes), lengths.strip()))
    for r, (ws, rk, local, worst, _, _) in enumerate(rows):
        assert (ws, rk, local) == (world, r, r)
        assert worst == max(elapsed)  # every rank sees the slowest rank's time
    # independent replicas: the ranks drew different request mixes
    assert rows[0][5] != rows[1][5]
    # whole-job throughput counts every rank's bytes over the slowest time
    per_rank = [row[4] for row in rows]
    assert R.aggregate_gbs(per_rank[0], 1, world, max(elapsed)) == pytest.approx(
        world * per_rank[0] / max(elapsed) / 1e9)
