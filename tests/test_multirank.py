"""Multi-GPU host logic on CPU: rank environment, per-rank inputs, max-over-ranks timing, whole-job
throughput, cost-balanced node sharding, and a real world_size-2 gloo process group.

Nodes are independent (the operator acts node by node in velocity space, paper Sec. 3), so the
path shards with no data-path collective; the only collectives are the timing ones.
"""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1809_10186_gb300 import multirank as MR
from paper_1809_10186_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_rank_env_defaults_and_torchrun_values():
    assert MR.rank_env({}) == MR.RankEnv(1, 0, 0)
    assert MR.rank_env({"WORLD_SIZE": "4", "RANK": "2", "LOCAL_RANK": "2"}) == MR.RankEnv(4, 2, 2)
    with pytest.raises(ValueError):
        MR.rank_env({"WORLD_SIZE": "2", "RANK": "2"})


def test_rank_seeds_give_distinct_reproducible_inputs():
    cfg = W.CONFIGS["vhs_n32"]
    a0, _ = W.two_maxwellian(3, 8, cfg["L"], MR.rank_seed(cfg["seed"], 0))
    a1, _ = W.two_maxwellian(3, 8, cfg["L"], MR.rank_seed(cfg["seed"], 1))
    b0, _ = W.two_maxwellian(3, 8, cfg["L"], MR.rank_seed(cfg["seed"], 0))
    assert np.array_equal(a0, b0)
    assert not np.allclose(a0, a1)


def test_job_throughput_is_whole_job_over_slowest_rank():
    assert MR.job_throughput(8, 2048, 5, 2.0) == pytest.approx(8 * 2048 * 5 / 2.0)
    with pytest.raises(ValueError):
        MR.job_throughput(1, 1, 1, 0.0)


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_nodes_contiguous_complete_balanced(world):
    # the ragged cavity mix: N in {16, 24, 32} with the workload's split, shuffled
    rng = np.random.default_rng(3)
    Ns = rng.choice([16, 24, 32], size=300, p=[0.4, 0.4, 0.2])
    costs = [MR.node_cost(int(n), 26, int(n)) for n in Ns]
    ranges = MR.shard_nodes(costs, world)
    assert len(ranges) == world
    assert ranges[0][0] == 0 and ranges[-1][1] == len(costs)
    for (s0, e0), (s1, e1) in zip(ranges, ranges[1:]):
        assert e0 == s1 and s0 <= e0
    total = sum(costs)
    worst = max(sum(costs[s:e]) for s, e in ranges)
    assert worst <= total / world + max(costs) * (1 + 1e-12)


def test_shard_nodes_equal_costs_split_evenly_and_edge_cases():
    assert MR.shard_nodes([1.0] * 10, 2) == [(0, 5), (5, 10)]
    assert MR.shard_nodes([], 3) == [(0, 0), (0, 0), (0, 0)]
    assert MR.shard_nodes([5.0], 2) in ([(0, 0), (0, 1)], [(0, 1), (1, 1)])
    with pytest.raises(ValueError):
        MR.shard_nodes([1.0], 0)


def test_node_cost_scales_with_grid_and_rule():
    assert MR.node_cost(32, 38, 32) / MR.node_cost(16, 38, 32) == pytest.approx(16.0)
    assert MR.node_cost(16, 26, 16) / MR.node_cost(16, 12, 16) == pytest.approx(13 / 6)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        # per-rank timing: the slowest rank defines the job's time
        t = MR.max_over_ranks(1.0 + 0.5 * rank, dist, "cpu")
        # every rank evaluates its own nodes (weak scaling) and derives the same job throughput
        value = MR.job_throughput(world, 16, 2, t)
        cfg = W.CONFIGS["vhs_n32"]
        f, _ = W.two_maxwellian(2, 8, cfg["L"], MR.rank_seed(cfg["seed"], rank))
        sig = torch.tensor([float(f.sum())], dtype=torch.float64)
        sigs = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(sigs, sig)
        # a shard plan computed independently on every rank is identical
        ranges = torch.tensor(MR.shard_nodes([1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0], world), dtype=torch.int64)
        allr = [torch.zeros_like(ranges) for _ in range(world)]
        dist.all_gather(allr, ranges)
        dist.barrier()
        out[rank] = (t, value, [float(x) for x in sigs], all(torch.equal(allr[0], r) for r in allr))
    finally:
        dist.destroy_process_group()


def test_world_size_two_gloo():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    assert sorted(out.keys()) == [0, 1]
    for r in range(world):
        t, value, sigs, same = out[r]
        assert t == pytest.approx(1.5)                       # max over ranks
        assert value == pytest.approx(world * 16 * 2 / 1.5)
        assert sigs[0] != sigs[1]                            # distinct inputs per rank
        assert same                                          # identical shard plans
    assert out[0][2] == out[1][2]


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"], env=env,
                       capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
