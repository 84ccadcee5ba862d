"""FP64 oracle references for the parity tests, computed in spawned worker processes.

Test infrastructure: the N = 32 workloads need the oracle on 16 or more nodes (about 1.5 s per
Q evaluation and 13 s per node for the derivative references, single-threaded), so the nodes are
spread over a pool of single-threaded processes. The pool uses the "spawn" start method: a
process forked after the parent has created a CUDA context can hang. Results are memoised per
session, so the precisions that share a workload share one set of references.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_CACHE: dict = {}
_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _inputs(cfg_name, kind):
    from paper_1809_10186_gb300 import workloads as W
    cfg = W.CONFIGS[cfg_name]
    F, _ = W.two_maxwellian(cfg["B"], cfg["N"], cfg["L"], cfg["seed"], dtype=np.float32)
    if kind == "grad":
        V = W.directions(cfg["B"], cfg["N"], cfg["seed"] + 100, dtype=np.float32)
        U = W.directions(cfg["B"], cfg["N"], cfg["seed"] + 200, dtype=np.float32)
        return cfg, F, V, U
    return cfg, F, None, None


def _job(args):
    """One worker's share: oracle values for the nodes `idx` of workload `cfg_name`."""
    import oracle as O
    kind, cfg_name, idx, rank = args
    cfg, F, V, U = _inputs(cfg_name, kind)
    op = O.OraclePlan(cfg["N"], cfg["L"], gamma=cfg["gamma"], M=cfg["M"], Nrho=cfg["Nrho"], nyquist="sym",
                      svd_rank=rank)
    out = {}
    for i in idx:
        f = F[i].astype(np.float64)
        if kind == "Q":
            out[i] = {"Q": O.fast_Q(op, f), "loss": np.real(O.loss_Q(op, f, f))}
        else:
            v, u = V[i].astype(np.float64), U[i].astype(np.float64)
            dop = O.dgamma_plan(op)
            out[i] = {"jvp": O.jvp(op, f, v), "jvp_loss": np.real(O.loss_Q(op, f, v) + O.loss_Q(op, v, f)),
                      "vjp": O.vjp(op, f, u), "dgamma": O.fast_Q(dop, f),
                      "dgamma_loss": np.real(O.loss_Q(dop, f, f))}
    return out


def references(kind, cfg_name, idx, rank=0, procs=None):
    """{node: {name: array}} for the nodes `idx`: kind "Q" gives Q and its loss term, kind "grad"
    the JVP along the workload's direction V, the VJP of U, dQ/dgamma and their loss parts."""
    key = (kind, cfg_name, tuple(idx), rank)
    if key in _CACHE:
        return _CACHE[key]
    procs = max(1, min(len(idx), procs or min(16, os.cpu_count() or 1)))
    old = {k: os.environ.get(k) for k in _THREAD_VARS}
    for k in _THREAD_VARS:
        os.environ[k] = "1"
    try:
        parts = [list(idx[i::procs]) for i in range(procs)]
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_job, [(kind, cfg_name, p, rank) for p in parts if p])
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    out = {}
    for r in res:
        out.update(r)
    _CACHE[key] = out
    return out


def sample_nodes(B, count, seed=5):
    """The first and last node and count - 2 others drawn without replacement (sorted)."""
    rng = np.random.default_rng(seed)
    rest = rng.choice(np.arange(1, B - 1), count - 2, replace=False)
    return sorted(set([0, B - 1] + [int(i) for i in rest]))


def batch_errors(got, ref, norm_ref=None):
    """Relative L2 errors over a batch: sqrt(sum_i |got_i - ref_i|^2) / sqrt(sum_i |n_i|^2) with
    n = ref (the |Q| normalisation) and, when given, n = norm_ref (e.g. the loss term |Q-|),
    plus the largest per-node ratios of both. got, ref, norm_ref: sequences of arrays."""
    d = np.array([np.linalg.norm(g - r) for g, r in zip(got, ref)])
    nq = np.array([np.linalg.norm(r) for r in ref])
    out = {"batch_q": float(np.sqrt((d * d).sum() / (nq * nq).sum())), "node_q": float((d / nq).max())}
    if norm_ref is not None:
        nl = np.array([np.linalg.norm(r) for r in norm_ref])
        out.update({"batch_loss": float(np.sqrt((d * d).sum() / (nl * nl).sum())), "node_loss": float((d / nl).max())})
    return out
