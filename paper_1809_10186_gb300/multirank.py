"""Host-side logic of multi-GPU runs: one process per GPU, nodes sharded with no collective.

Nodes are independent (the collision operator acts in velocity space only, node by node, paper
Sec. 3), so a multi-GPU run gives every rank its own nodes and needs no data-path exchange. The
only collectives are the timing ones: a barrier around the timed region and the maximum of the
ranks' times (the slowest rank defines the whole job's time).

Everything here is independent of the GPU and is tested with the gloo backend on CPU.
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass(frozen=True)
class RankEnv:
    world: int
    rank: int
    local: int


def rank_env(environ=None) -> RankEnv:
    """WORLD_SIZE / RANK / LOCAL_RANK as set by torchrun (1 / 0 / 0 when absent)."""
    env = os.environ if environ is None else environ
    world = int(env.get("WORLD_SIZE", "1"))
    rank = int(env.get("RANK", "0"))
    local = int(env.get("LOCAL_RANK", str(rank)))
    if world < 1 or not (0 <= rank < world) or local < 0:
        raise ValueError("inconsistent rank environment: WORLD_SIZE=%d RANK=%d LOCAL_RANK=%d" % (world, rank, local))
    return RankEnv(world, rank, local)


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of a rank's synthetic inputs under weak scaling: distinct per rank, reproducible."""
    return int(base_seed) + int(rank)


def max_over_ranks(x: float, dist=None, device: str = "cpu") -> float:
    """Maximum of a per-rank scalar over all ranks (the identity without a process group)."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, nodes_per_rank: int, steps: int, seconds: float) -> float:
    """Whole-job node evaluations per second under weak scaling: every rank evaluates
    nodes_per_rank nodes per step, and the job takes the slowest rank's time."""
    if seconds <= 0.0:
        raise ValueError("elapsed time must be positive")
    return world * nodes_per_rank * steps / seconds


def node_cost(N: int, M: int, N_rho: int) -> float:
    """Relative cost of one node: the translates dominate, N_rho (M/2) 12 N^4 flops."""
    return float(N_rho) * (M // 2) * 12.0 * float(N) ** 4


def shard_nodes(costs, world: int):
    """Contiguous node ranges [start, end) per rank, balanced by per-node cost.

    For a caller that shards one batch (strong scaling). Rank k's range ends at the first node
    whose cost prefix reaches (k + 1) / world of the total, so every node is in exactly one range
    and the ranges are in node order; the largest range cost exceeds total / world by at most one
    node's cost.
    """
    costs = [float(c) for c in costs]
    if world < 1:
        raise ValueError("world must be >= 1")
    if any(c < 0 for c in costs):
        raise ValueError("costs must be non-negative")
    total = sum(costs)
    bounds = [0]
    prefix = 0.0
    i = 0
    n = len(costs)
    for k in range(1, world):
        target = total * k / world
        while i < n and prefix + costs[i] <= target + 1e-12 * total:
            prefix += costs[i]
            i += 1
        # put the straddling node on whichever side keeps the boundary closer to the target
        if i < n and (target - prefix) > (prefix + costs[i] - target):
            prefix += costs[i]
            i += 1
        bounds.append(i)
    bounds.append(n)
    return [(bounds[k], bounds[k + 1]) for k in range(world)]
