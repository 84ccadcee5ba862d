#!/usr/bin/env python
"""Throughput of batched Q(f, f) on the N = 32 VHS workload (node evaluations per second).

Workload ("vhs_n32"): 2048 DG nodes per GPU, each a seeded two-Maxwellian mixture on an
N = 32 grid over [-7, 7]^3; VHS omega = 0.74 (gamma = 0.52); N_rho = 32 Gauss-Legendre
radial points on [0, R], R = 4L/(3 + sqrt 2); M = 38 sphere points (19 antipodal pairs);
radial kernel SVD-truncated at 1e-8. One step = one dgfs_collide over the whole batch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec f16s|bf16s|fp32]
  python bench.py --impl reference ...      # the FP64 CPU oracle on the host cores

Multi-GPU (torchrun, one process per GPU): nodes are independent, every rank evaluates its
own 2048 nodes (weak scaling) and no data-path collective is used; the timed region is
bracketed by barriers and the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Q(f,f) node-evals/s at N=32 VHS, % roofline, mixed-prec vs FP32 at stated err"
WORKLOAD = "vhs_n32"
# Tolerances of the relative L2 error against the FP64 oracle, over the sampled nodes as one
# vector, normalised by ||Q|| and by the loss term ||Q-||. At this workload F16S is held to the
# 1e-3 of ||Q|| stated for the split 16-bit forms (the tests allow 1e-2 on rougher inputs); BF16S
# keeps its own wider tolerance (it does not reach 1e-3).
TOL_Q = {"fp64": 1e-10, "fp32": 1e-5, "f16s": 1e-3, "bf16s": 5e-2, "f16x3": 1e-5, "bf16x3": 1e-3}
TOL_L = {"fp64": 1e-10, "fp32": 1e-5, "f16s": 1e-3, "bf16s": 5e-3, "f16x3": 1e-5, "bf16x3": 1e-4}
MODES = ("fp32", "f16s", "bf16s", "f16x3", "bf16x3")
DTYPES = {"fp32": "f32", "fp64": "f64", "f16s": "f16 data, f16 hi+lo filters, f32 accumulate",
          "bf16s": "bf16 data, bf16 hi+lo filters, f32 accumulate",
          "f16x3": "f16 hi+lo data and filters (3 products), f32 accumulate",
          "bf16x3": "bf16 hi+lo data and filters (3 products), f32 accumulate"}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="f16s", choices=["fp32", "f16s", "bf16s", "f16x3", "bf16x3"],
                    help="f16s: tensor-core translates, fp16 data + split fp16 filters; f16x3 / bf16x3: data and "
                         "filters split (three products)")
    ap.add_argument("--nodes", type=int, default=None, help="nodes per GPU (default 2048)")
    ap.add_argument("--chunk", type=int, default=0,
                    help="nodes per internal chunk (plan max_batch); 0: the whole per-GPU batch in one chunk")
    ap.add_argument("--sphere", type=int, default=0, choices=[0, 6, 12, 26, 38],
                    help="sphere rule size M of the headline leg (0: the workload's 38); smaller rules "
                         "give the translate kernel's fixed cost per CTA by a fit over M")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--dg", action="store_true",
                    help="measure the DG element collision term (Sec. 3.4, SVD variant) on the 1-D slab "
                         "workload instead of the headline (prints its own line)")
    ap.add_argument("--vss", action="store_true",
                    help="VSS kernel (alpha = 1.40, argon) on 256 nodes of N = 32, FP32, instead of the headline")
    ap.add_argument("--grad", action="store_true",
                    help="grad_n32: JVP, VJP and dQ/dgamma throughput on 512 nodes of N = 32, FP32")
    ap.add_argument("--ragged", action="store_true",
                    help="cavity_ragged: 9216 nodes of mixed N (16/24/32) through one graph-captured ragged schedule")
    ap.add_argument("--slab", action="store_true",
                    help="1-D DGFS Fourier heat transfer (10 elements x 3 nodes, N = 24) SSP-RK2 steps")
    ap.add_argument("--slab-profile", type=int, default=0,
                    help="with --slab: run this many more steps and report the temperature profile")
    ap.add_argument("--rk", type=int, default=0, choices=[0, 2, 3],
                    help="measure SSP-RK2/3 time steps (dgfs_ssprk) of the headline workload instead "
                         "(prints its own line)")
    ap.add_argument("--oracle-worker", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


# ---- CPU oracle leg (the only place bench.py runs oracle/) ---------------------------------

def _oracle_job(args):
    """Runs in a spawned worker: Q of the given nodes with the FP64 oracle (unchanged)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import numpy as np
    import oracle as O
    from paper_1809_10186_gb300 import workloads as W
    cfg = W.CONFIGS[WORKLOAD]
    idx, B, seed, rank = args
    F, _ = W.two_maxwellian(B, cfg["N"], cfg["L"], seed, dtype=np.float32)
    plan = O.OraclePlan(cfg["N"], cfg["L"], gamma=cfg["gamma"], M=cfg["M"], Nrho=cfg["Nrho"],
                        nyquist="sym", svd_rank=rank)
    out = []
    t0 = time.perf_counter()
    for i in idx:
        Fi = F[i].astype(np.float64)
        q = O.fast_Q(plan, Fi)
        loss = np.real(O.loss_Q(plan, Fi, Fi))
        out.append((i, q, loss))
    return out, time.perf_counter() - t0


def oracle_sample(nodes_idx, B, seed, rank, procs):
    """Evaluate the oracle on `nodes_idx` with `procs` single-threaded spawned workers."""
    import multiprocessing as mp
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        chunks = [nodes_idx[i::procs] for i in range(procs) if nodes_idx[i::procs]]
        with ctx.Pool(len(chunks)) as pool:
            # plan construction happens inside each job; the timed part is reported per job
            t0 = time.perf_counter()
            res = pool.map(_oracle_job, [(c, B, seed, rank) for c in chunks])
            wall = time.perf_counter() - t0
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    results = [r for part, _ in res for r in part]
    compute_wall = max(t for _, t in res)       # slowest worker's evaluation time
    return results, compute_wall, wall, len(chunks)


# ---- clocks during the timed region ----------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            v = [x.strip() for x in line.split(",")]
            if len(v) < 9:
                continue
            try:
                sm.append(float(v[1]))
                smax.append(float(v[2]))
            except ValueError:
                continue
            for n, flag in zip(names, v[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---- roofline bookkeeping ----------------------------------------------------------------------

def translate_flops_per_node(N, Nrho, npairs, prec):
    """Flops the chosen formulation executes in the translate-product step, per node.

    Tensor-core modes: per (radial point, pair) two 3-D translates, each three dense N x N
    circulant passes over N^2 lines (2 N^4 flops per pass), every filter split into hi + lo parts
    (two products per contraction; three, hi hi + hi lo + lo hi, when the data are split too), then
    the product and weighted accumulation (3 N^3).
    FP32 / FP64 (N = 8, 16, 32): translates in Fourier space, one complex 3-D inverse transform per
    (radial point, pair) (radix-2: 5 N^3 log2 N^3) giving both translates, plus ~17 flops per
    point of phases, product and accumulation.
    """
    if prec in ("fp32", "fp64") and N in (8, 16, 32):
        return Nrho * npairs * (5.0 * N ** 3 * math.log2(N ** 3) + 17.0 * N ** 3)
    mma = 12.0 * N ** 4
    elem = 3.0 * N ** 3
    mult = {"fp32": 1, "fp64": 1, "f16s": 2, "bf16s": 2, "f16x3": 3, "bf16x3": 3}[prec]
    return Nrho * npairs * (mult * mma + elem)


def shape_ceiling_fields(N, Nr, npairs, prec, measured, launch_ms, nodes, clocks):
    """The kernel's cycles per (radial point, pair) step and SM (launch time at the sampled SM clock)
    against mma_shape_ceiling: how close the kernel runs to what its MMA shapes allow."""
    ceil, ctas = mma_shape_ceiling(N, prec, measured.get("mma_cycles", {}))
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz")
    if not ceil or not mhz or not nodes:
        return {}
    kernel = launch_ms / 1e3 * mhz * 1e6 * measured["sms"] / (nodes * Nr * npairs * ctas)
    return {"mma_shape_cycles_per_step": ceil, "kernel_cycles_per_step": kernel,
            "frac_of_mma_shape_ceiling": ceil / kernel,
            "mma_shape_basis": "cycles per (radial point, pair) step and SM that the kernel's own MMAs need back "
                               "to back at the measured rates of their shapes (peaks_measured.mma_cycles), "
                               "against the kernel's cycles per step at the sampled SM clock"}


def mma_shape_ceiling(N, prec, mma):
    """Cycles per (radial point, pair) step and SM that the translate kernel's own MMAs need when
    issued back to back at the measured rates of their shapes (M = 128, K = 16), and the CTAs that
    share one step. F16S / BF16S (one CTA per step, T = N^2 / 128 tiles, N / 16 K steps): pass 1 two
    MMAs (hi, lo) of N = 2n per K step with A in TMEM, passes 2 and 3 one MMA of N = 2n per sign and
    K step with A in shared memory. F16X3 / BF16X3 (a CTA pair per step, T / 2 tiles each): pass 1
    one MMA of N = 4n and one of N = 2n (A in TMEM), passes 2 and 3 per sign one of N = 2n and one of
    N = n (A in shared memory). None for the CUDA-core precisions or a missing shape."""
    T, ks = N * N // 128, N // 16
    try:
        if prec in ("f16s", "bf16s"):
            return T * ks * 2 * mma["tmem_n%d" % (2 * N)] + 2 * T * 2 * ks * mma["smem_n%d" % (2 * N)], 1
        if prec in ("f16x3", "bf16x3"):
            th = T // 2
            return (th * ks * (mma["tmem_n%d" % (4 * N)] + mma["tmem_n%d" % (2 * N)]) +
                    2 * th * 2 * ks * (mma["smem_n%d" % (2 * N)] + mma["smem_n%d" % N])), 2
    except KeyError:
        return None, None
    return None, None


def fft_algorithmic_flops_per_node(N, Nrho, npairs):
    """The method's work counted with radix-2 FFTs (one complex 3-D IDFT per pair gives both
    real translates; 5 N^3 log2 N^3 flops) plus ~20 flops per point per pair of phase,
    product and accumulation."""
    return Nrho * npairs * (5.0 * N ** 3 * math.log2(N ** 3) + 20.0 * N ** 3)


# DRAM bytes (read + write) per node of one translate-product launch at N = 32, N_rho = 32, M = 38,
# from the ncu capture of a 512-node launch summarised in profiles/ (None for configurations
# without a capture of the current kernel version).
TRAFFIC_PER_NODE = {("f16s", 32, 32, 38): (180026368 + 2091159552) / 512, ("bf16s", 32, 32, 38): (185963520 + 2090830592) / 512,
                    ("f16x3", 32, 32, 38): (109169920 + 2091046656) / 512,
                    ("fp32", 32, 32, 38): None}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def measure_peaks():
    """Peaks measured on this device for the rooflines: SM count and L2 size (device properties),
    the FP32 and FP64 FMA rates of the CUDA cores (dgfs_device_fma_peaks: independent FMA chains
    on every SM), and dense matmul rates through cuBLAS (torch.matmul of 8192^3 fp16, bf16 and
    TF32 operands, best of 5 after a warm-up; 2 n^3 flops). Changes no device setting."""
    import torch
    from paper_1809_10186_gb300 import binding
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    fp32, fp64 = binding.device_fma_peaks()

    def mm(dtype, tf32=False):
        n = 8192
        g = torch.Generator(device="cuda").manual_seed(0)
        a = torch.randn(n, n, device="cuda", dtype=dtype, generator=g)
        b = torch.randn(n, n, device="cuda", dtype=dtype, generator=g)
        old = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = tf32
        try:
            torch.matmul(a, b)
            torch.cuda.synchronize()
            best = None
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
        finally:
            torch.backends.cuda.matmul.allow_tf32 = old
        del a, b
        return 2.0 * n ** 3 / (best / 1e3) / 1e12

    # cycles per back-to-back tcgen05 MMA (M = 128, K = 16) of the shapes the translate kernels issue
    mma = {"smem_n%d" % n: binding.device_mma_cycles(n, False) for n in (32, 64, 128, 256)}
    mma.update({"tmem_n%d" % n: binding.device_mma_cycles(n, True) for n in (64, 128, 256)})
    out = {"sms": props.multi_processor_count,
           "l2_bytes": getattr(props, "L2_cache_size", None),
           "fp32_fma_tflops": fp32, "fp64_fma_tflops": fp64,
           "fp16_dense_tflops": mm(torch.float16), "bf16_dense_tflops": mm(torch.bfloat16),
           "tf32_dense_tflops": mm(torch.float32, tf32=True),
           "mma_cycles": mma,
           "how": "FMA chains on every SM (libdgfs probe); cuBLAS 8192^3 matmuls, best of 5 (burst); "
                  "cycles per back-to-back tcgen05.mma kind::f16, M = 128, K = 16, A from shared memory or "
                  "TMEM (libdgfs probe, slowest SM)"}
    torch.cuda.empty_cache()
    return out


def accuracy_of(q_modes, res):
    """Errors of every mode's result against the oracle sample `res` [(node, Q, loss)]: the relative
    L2 error of the sampled nodes as one vector by ||Q|| and by ||Q-||, the largest per-node values,
    the mass drift, and whether the mode meets its tolerance."""
    import numpy as np
    acc = {}
    for mode, qm in q_modes.items():
        qc = qm.double().cpu().numpy()
        d, nq, nl, mass = [], [], [], []
        for i, qo, loss in res:
            d.append(np.linalg.norm(qc[i] - qo))
            nq.append(np.linalg.norm(qo))
            nl.append(np.linalg.norm(loss))
            mass.append(abs(qc[i].sum()) / np.abs(loss).sum())
        d, nq, nl = map(np.array, (d, nq, nl))
        bq = float(np.sqrt((d * d).sum() / (nq * nq).sum()))
        bl = float(np.sqrt((d * d).sum() / (nl * nl).sum()))
        acc[mode] = {"rel_l2_vs_Q": bq, "rel_l2_vs_loss": bl,
                     "node_max_vs_Q": float((d / nq).max()), "node_max_vs_loss": float((d / nl).max()),
                     "mass_drift_max": float(max(mass)),
                     "tolerance_vs_Q": TOL_Q.get(mode), "tolerance_vs_loss": TOL_L.get(mode),
                     "meets_tolerance": bool(bq < TOL_Q.get(mode, 0) and bl < TOL_L.get(mode, 0))}
    return acc


def equal_accuracy(values, acc):
    """For each stated error level, the modes whose batch errors (by ||Q|| and ||Q-||) are within it,
    their node-evals/s, and the fastest of them against FP32 when FP32 is among them."""
    out = {}
    for level in (1e-5, 1e-3):
        ok = {m: values[m] for m in values if m in acc and acc[m]["rel_l2_vs_Q"] < level
              and acc[m]["rel_l2_vs_loss"] < level}
        if not ok:
            continue
        best = max(ok, key=ok.get)
        row = {"modes": ok, "fastest": best}
        if "fp32" in ok:
            row["fastest_over_fp32"] = ok[best] / ok["fp32"]
        out["%g" % level] = row
    return out


# ---- the reference arm: the FP64 CPU oracle ----------------------------------------------------

def run_reference(a):
    import numpy as np  # noqa: F401
    from paper_1809_10186_gb300.multirank import rank_env
    env = rank_env()
    world = env.world
    if env.rank != 0:   # rank 0 alone runs the oracle; the other ranks exit without work
        return 0
    from paper_1809_10186_gb300 import workloads as W
    cfg = W.CONFIGS[WORKLOAD]
    cores = os.cpu_count() or 1
    B = cfg["B"]
    per_step = max(1, min(cores, 16))
    times = []
    total = 0
    node = 0
    for step in range(a.warmup + a.steps):
        idx = [(node + i) % B for i in range(per_step)]
        node += per_step
        _, comp, _, procs = oracle_sample(idx, B, cfg["seed"], 0, per_step)
        if step >= a.warmup:
            times.append(comp)
            total += len(idx)
    val = total / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "node-evals/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "%s: 2048-node batch, sampled %d nodes per step" % (WORKLOAD, per_step),
                       "N": cfg["N"], "M": cfg["M"], "N_rho": cfg["Nrho"], "nodes_per_step": per_step},
            "cpu_baseline": {"value": val, "unit": "node-evals/s", "cores": procs, "kind": "oracle",
                             "sample": "%d nodes per step, one single-threaded process per node" % per_step},
            "e2e": {"value": val, "unit": "node-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---- our arm -----------------------------------------------------------------------------------

def run_dg(a):
    """DG element collision term of the slab workload: 16 elements x K = 3 Gauss-Lobatto nodes,
    N = 24, omega = 0.81, M = 12, FP32; C[e][m] = sum_r Q(f_r, g_r) (every R_m = 3 at svd_tol 0),
    evaluated as sign(lambda_r) Q(f_r, f_r) since every slice H[m] is symmetric."""
    import numpy as np
    import torch
    from paper_1809_10186_gb300 import binding, workloads as W
    torch.cuda.set_device(0)
    cfg = W.CONFIGS["slab_n24"]
    N, L, K = cfg["N"], cfg["L"], 3
    E = cfg["B"] // K
    F, _ = W.two_maxwellian(E * K, N, L, cfg["seed"], dtype=np.float32)
    f = torch.from_numpy(F.reshape(E, K, N, N, N)).cuda()
    plan = binding.Plan(N=N, L=L, gamma=cfg["gamma"], M=cfg["M"], N_rho=cfg["Nrho"], precision="fp32",
                        max_batch=E * K * K)
    _, _, H = binding.host_dg_tensor(K)
    dg = binding.DGElement(plan, H, max_elements=E)
    c = torch.empty_like(f)
    for _ in range(a.warmup):
        dg.collide(f, out=c)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    plan.profile_begin()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        dg.collide(f, out=c)
    e1.record()
    torch.cuda.synchronize()
    prof = plan.profile_end()
    clocks = sampler.stop()
    plan.stream_status()
    ms = e0.elapsed_time(e1) / a.steps
    line = {"metric": "DG element collision terms/s, 1-D slab (16 elements x 3 nodes, N=24, omega=0.81, M=12)",
            "value": E / (ms / 1e3), "unit": "elements/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "Q_evals_per_s": E * dg.total_rank / (ms / 1e3),
            "config": {"workload": "slab_n24 DG element term, SVD variant", "elements": E, "K": K,
                       "ranks": dg.ranks, "N": N, "M": cfg["M"], "N_rho": cfg["Nrho"]},
            "gpu_launches": prof["launches"], "clocks": clocks}
    print(json.dumps(line))
    dg.close()
    plan.close()
    return 0


def run_rk(a):
    """Space-homogeneous SSP-RK steps (eqs. SSPRK2/3) of the headline workload's 2048 nodes: each
    step is `order` collision evaluations plus the stage kernels, all through dgfs_ssprk."""
    import numpy as np
    import torch
    from paper_1809_10186_gb300 import binding, workloads as W
    torch.cuda.set_device(0)
    cfg = W.CONFIGS[WORKLOAD]
    N, L, B = cfg["N"], cfg["L"], a.nodes or cfg["B"]
    F, _ = W.two_maxwellian(B, N, L, cfg["seed"], dtype=np.float32)
    f = torch.from_numpy(F).cuda()
    plan = binding.Plan(N=N, L=L, gamma=cfg["gamma"], M=cfg["M"], N_rho=cfg["Nrho"], svd_tol=cfg["svd_tol"],
                        precision=a.prec, max_batch=B)
    plan.ssprk(f, 0.01, a.warmup, order=a.rk)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    plan.profile_begin()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.ssprk(f, 0.01, a.steps, order=a.rk)
    e1.record()
    torch.cuda.synchronize()
    prof = plan.profile_end()
    clocks = sampler.stop()
    plan.stream_status()
    ms = e0.elapsed_time(e1) / a.steps
    mom = plan.moments(f).cpu().numpy()
    line = {"metric": "SSP-RK%d node-steps/s, space-homogeneous, N=32 VHS" % a.rk, "value": B / (ms / 1e3),
            "unit": "node-steps/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
            "higher_is_better": True, "dtype": a.prec, "data": "synthetic",
            "config": {"workload": "%s: %d nodes, dt = 0.01" % (WORKLOAD, B), "order": a.rk},
            "mass_after": float(mom[:, 0].mean()), "gpu_launches": prof["launches"], "clocks": clocks}
    print(json.dumps(line))
    plan.close()
    return 0


def vss_flops_per_node(N, Nrho, npairs):
    """Radix-2 count of the VSS gain per node: per radial and sphere point one complex 3-D inverse
    transform (both translates) and half a forward one (two sphere points per transform), plus
    ~20 flops per point of phases, products, Hermitian separation and accumulation."""
    return Nrho * npairs * (7.5 * N ** 3 * math.log2(N ** 3) + 20.0 * N ** 3)


def run_vss(a):
    """Q(f, f) for the VSS kernel (eq. B_gen, alpha != 1) on the vss_n32 workload, FP32."""
    import numpy as np
    import torch
    from paper_1809_10186_gb300 import binding, workloads as W
    torch.cuda.set_device(0)
    cfg = W.CONFIGS["vss_n32"]
    N, L, B = cfg["N"], cfg["L"], a.nodes or cfg["B"]
    F, _ = W.two_maxwellian(B, N, L, cfg["seed"], dtype=np.float32)
    f = torch.from_numpy(F).cuda()
    q = torch.empty_like(f)
    plan = binding.Plan(N=N, L=L, gamma=cfg["gamma"], alpha=cfg["alpha"], M=cfg["M"], N_rho=cfg["Nrho"],
                        precision="fp32", max_batch=B)
    npairs = plan.info["n_pairs"]
    for _ in range(a.warmup):
        plan.collide(f, out=q)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    plan.profile_begin()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        plan.collide(f, out=q)
    e1.record()
    torch.cuda.synchronize()
    prof = plan.profile_end()
    clocks = sampler.stop()
    plan.stream_status()
    ms = e0.elapsed_time(e1) / a.steps
    value = B / (ms / 1e3)
    flops = vss_flops_per_node(N, cfg["Nrho"], npairs)
    from paper_1809_10186_gb300 import binding as _b
    peak = _b.device_fma_peaks()[0]
    line = {"metric": "Q(f,f) node-evals/s at N=32 VSS (alpha=1.40, omega=0.81), FP32", "value": value,
            "unit": "node-evals/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "vss_n32: %d two-Maxwellian nodes, N=32 on [-7,7]^3, N_rho=32, M=38" % B,
                       "alpha": cfg["alpha"], "N": N, "M": cfg["M"], "N_rho": cfg["Nrho"],
                       "chunk_nodes": plan.info["chunk_nodes"],
                       "workspace_gb": round(plan.info["workspace_bytes"] / 2 ** 30, 2),
                       "l2": "no flush: translate spectra of a transform batch exceed L2"},
            "roofline": {"bound": "alu", "scope": "whole VSS step (transforms and elementwise kernels)",
                         "achieved": flops * value / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops * value / 1e12 / peak, "traffic": None, "flops_per_node": flops,
                         "peak_source": "measured FP32 FMA rate of this GPU (of measured)"},
            "gpu_launches": prof["launches"], "clocks": clocks}
    print(json.dumps(line))
    plan.close()
    return 0


def run_grad(a):
    """Tangent and adjoint of Q(f, f) on the grad_n32 workload (512 two-Maxwellian nodes, N = 32,
    omega = 0.81, M = 38, FP32): node-evals/s of dgfs_collide_jvp, dgfs_collide_vjp and
    dgfs_collide_dgamma, each timed over `steps` calls."""
    import numpy as np
    import torch
    from paper_1809_10186_gb300 import binding, workloads as W
    torch.cuda.set_device(0)
    cfg = W.CONFIGS["grad_n32"]
    N, L, B = cfg["N"], cfg["L"], cfg["B"]
    F, _ = W.two_maxwellian(B, N, L, cfg["seed"], dtype=np.float32)
    D = W.directions(B, N, cfg["seed"] + 1, dtype=np.float32)
    f, v = torch.from_numpy(F).cuda(), torch.from_numpy(D).cuda()
    out = torch.empty_like(f)
    plan = binding.Plan(N=N, L=L, gamma=cfg["gamma"], M=cfg["M"], N_rho=cfg["Nrho"], precision="fp32", max_batch=B)
    calls = {"jvp": lambda: plan.collide_jvp(f, v, out=out), "vjp": lambda: plan.collide_vjp(f, v, out=out),
             "dgamma": lambda: plan.collide_dgamma(f, out=out), "collide": lambda: plan.collide(f, out=out)}
    res = {}
    sampler = ClockSampler(0)
    sampler.start()
    for name, call in calls.items():
        for _ in range(a.warmup):
            call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.steps):
            call()
        e1.record()
        torch.cuda.synchronize()
        res[name] = B / (e0.elapsed_time(e1) / a.steps / 1e3)
    # the JVP and Q(f, f) of tensor-core plans (translates on the tensor cores; the JVP by polarisation)
    tc = {}
    for prec in ("f16x3", "f16s"):
        pt = binding.Plan(N=N, L=L, gamma=cfg["gamma"], M=cfg["M"], N_rho=cfg["Nrho"], precision=prec, max_batch=B)
        tc[prec] = {}
        for name, call in (("jvp", lambda: pt.collide_jvp(f, v, out=out)), ("collide", lambda: pt.collide(f, out=out))):
            for _ in range(a.warmup):
                call()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(a.steps):
                call()
            e1.record()
            torch.cuda.synchronize()
            tc[prec][name] = B / (e0.elapsed_time(e1) / a.steps / 1e3)
        pt.stream_status()
        pt.close()
    clocks = sampler.stop()
    plan.stream_status()
    line = {"metric": "VJP node-evals/s (dQ(f,f)/df transposed), N=32 VHS omega=0.81, M=38, FP32", "value": res["vjp"],
            "unit": "node-evals/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "grad_n32: %d nodes, unit-norm Gaussian directions" % B, "N": N, "M": cfg["M"],
                       "N_rho": cfg["Nrho"]},
            "jvp": res["jvp"], "vjp": res["vjp"], "dgamma": res["dgamma"], "collide": res["collide"],
            "tensor_core_plans": tc, "clocks": clocks}
    print(json.dumps(line))
    plan.close()
    return 0


def run_ragged(a):
    """The ragged cavity mesh: 9216 near-equilibrium nodes, N in {16, 24, 32} (40/40/20 %), per-node
    VHS omega in {0.5, 0.74, 0.81}, M = 26; one plan per N in the --prec mode (every tensor-core
    precision takes N = 24 on the 32-point tiles), all classes in one dgfs_ragged schedule captured
    as one CUDA graph and replayed."""
    import numpy as np
    import torch
    from paper_1809_10186_gb300 import binding, workloads as W
    torch.cuda.set_device(0)
    cfg = W.CONFIGS["cavity_ragged"]
    Ns, L, M, B = cfg["Ns"], cfg["L"], cfg["M"], cfg["B"]
    node_N, node_omega = W.ragged_layout(B, Ns, cfg["split"], cfg["omegas"], cfg["seed"])
    offs = np.zeros(B, np.int64)
    offs[1:] = np.cumsum(node_N.astype(np.int64) ** 3)[:-1]
    packed = np.empty(int(offs[-1] + int(node_N[-1]) ** 3), np.float32)
    for n in Ns:
        idx = np.nonzero(node_N == n)[0]
        fields = W.near_equilibrium(len(idx), n, L, cfg["seed"] + n, dtype=np.float32)
        for j, i in enumerate(idx):
            packed[offs[i]:offs[i] + n ** 3] = fields[j].ravel()
    gam = 2.0 * (1.0 - node_omega)
    bb = 1.0 / (2.0 ** (3.0 - node_omega) * np.array([math.gamma(2.5 - w) for w in node_omega]) * math.pi)
    precs = {n: a.prec for n in Ns}
    plans = [binding.Plan(N=n, L=L, M=M, N_rho=n, precision=precs[n]) for n in Ns]
    cls = [list(Ns).index(int(n)) for n in node_N]
    sched = binding.RaggedSchedule(plans, cls, offs, node_gamma=gam, node_b=bb)
    x = torch.from_numpy(packed).cuda()
    y = torch.empty_like(x)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        for _ in range(max(1, a.warmup)):
            sched.collide(x, out=y, stream=st)
    torch.cuda.current_stream().wait_stream(st)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        sched.collide(x, out=y, stream=st)
    g.replay()
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    for p in plans:
        p.stream_status()
    ms = e0.elapsed_time(e1) / a.steps
    line = {"metric": "ragged Q(f,f) node-evals/s, cavity mesh 9216 nodes, N in {16,24,32}, one CUDA graph",
            "value": B / (ms / 1e3), "unit": "node-evals/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms, "higher_is_better": True, "dtype": ",".join("N=%d:%s" % (n, precs[n]) for n in Ns),
            "data": "synthetic",
            "config": {"workload": "cavity_ragged: %d nodes, split %s, omegas %s, M=%d, N_rho=N" % (
                B, cfg["split"], cfg["omegas"], M), "nodes_per_N": {int(n): int(np.sum(node_N == n)) for n in Ns}},
            "clocks": clocks}
    print(json.dumps(line))
    sched.close()
    for p in plans:
        p.close()
    return 0


def run_slab(a):
    """SSP-RK2 steps of the 1-D DGFS solver on the Fourier heat-transfer setup: every step is two
    right-hand sides, each the DG element collision term of the 10 elements (90 bilinear Q at N = 24)
    plus the transport kernels, and the stage combinations."""
    import numpy as np
    import torch
    from paper_1809_10186_gb300 import binding, workloads as W
    torch.cuda.set_device(0)
    cfg = W.CONFIGS["fourier_slab"]
    N, L, K, I = cfg["N"], cfg["L"], cfg["K"], cfg["I"]
    edges = np.linspace(0.0, 1.0, I + 1)
    plan = binding.Plan(N=N, L=L, gamma=cfg["gamma"], M=cfg["M"], N_rho=cfg["Nrho"], precision=cfg["prec"],
                        max_batch=I * K * K)
    slab = binding.Slab(plan, K, edges, cfg["Kn"], (0, 0, 0, cfg["T_left"]), (0, 0, 0, cfg["T_right"]))
    c = W.velocity_grid(N, L)
    cx, cy, cz = np.meshgrid(c, c, c, indexing="ij")
    f0 = (np.pi ** -1.5 * np.exp(-(cx ** 2 + cy ** 2 + cz ** 2))).astype(np.float32)
    F = torch.from_numpy(np.broadcast_to(f0, (I, K, N, N, N)).copy()).cuda()
    # kernels of one step, counted by the plan's profiler on an eager step of a scratch copy (a
    # profiling plan steps eagerly; the timed steps replay the step's captured graph)
    G = F.clone()
    plan.profile_begin()
    slab.ssprk(G, cfg["dt"], 1)
    torch.cuda.synchronize()
    per_step = plan.profile_end()["launches"]
    del G
    slab.ssprk(F, cfg["dt"], a.warmup)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    slab.ssprk(F, cfg["dt"], a.steps)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    plan.stream_status()
    ms = e0.elapsed_time(e1) / a.steps
    line = {"metric": "1-D DGFS SSP-RK2 steps/s, Fourier heat transfer (10 elements x 3 nodes, N=24, M=12)",
            "value": 1e3 / ms, "unit": "steps/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "phase_space_updates_per_s": I * K * N ** 3 / (ms / 1e3),
            "config": {"workload": "fourier_slab: walls %.4f / %.4f, Kn %.4f, dt %g" % (
                cfg["T_left"], cfg["T_right"], cfg["Kn"], cfg["dt"]), "I": I, "K": K, "N": N, "M": cfg["M"],
                "launch": "one step captured as a CUDA graph, replayed"},
            "gpu_launches": per_step * a.steps, "clocks": clocks}
    if a.slab_profile:
        slab.ssprk(F, cfg["dt"], a.slab_profile)
        mom = plan.moments(F.reshape(I * K, N, N, N)).cpu().numpy()
        xs = (0.5 * (edges[:-1, None] + edges[1:, None]) + 0.5 * np.diff(edges)[:, None]
              * np.array([-1.0, 0.0, 1.0])[None, :]).ravel()
        line["temperature_profile"] = {"t": cfg["dt"] * (a.warmup + a.steps + a.slab_profile),
                                       "x": [round(float(x), 4) for x in xs],
                                       "T_kelvin": [round(float(t) * 273.0, 2) for t in mom[:, 4]],
                                       "n": [round(float(v), 5) for v in mom[:, 0]]}
    print(json.dumps(line))
    slab.close()
    plan.close()
    return 0


def main():
    a = _args()
    if a.oracle_worker:
        return 0
    if a.impl == "reference":
        return run_reference(a)
    if a.dg:
        return run_dg(a)
    if a.rk:
        return run_rk(a)
    if a.vss:
        return run_vss(a)
    if a.slab:
        return run_slab(a)
    if a.ragged:
        return run_ragged(a)
    if a.grad:
        return run_grad(a)
    import numpy as np
    import torch
    from paper_1809_10186_gb300 import binding, workloads as W
    from paper_1809_10186_gb300.multirank import job_throughput, max_over_ranks, rank_env, rank_seed

    env = rank_env()
    world, rank, local = env.world, env.rank, env.local
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    binding.lib()

    cfg = W.CONFIGS[WORKLOAD]
    N, L, M, Nr = cfg["N"], cfg["L"], a.sphere or cfg["M"], cfg["Nrho"]
    B = a.nodes or cfg["B"]
    prec = a.prec
    F, _ = W.two_maxwellian(B, N, L, rank_seed(cfg["seed"], rank), dtype=np.float32)
    f = torch.from_numpy(F).cuda()
    q = torch.empty_like(f)
    plan = binding.Plan(N=N, L=L, gamma=cfg["gamma"], M=M, N_rho=Nr, svd_tol=cfg["svd_tol"], precision=prec,
                        max_batch=a.chunk if a.chunk > 0 else B)
    npairs = plan.info["n_pairs"]
    # the autotuner picks radial points per CTA and nodes per chunk on this batch (outside the timed region)
    tuning = {prec: plan.autotune(f)}

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(p, steps, warmup):
        for _ in range(warmup):
            p.collide(f, out=q)
        barrier()
        sampler = ClockSampler(local)
        sampler.start()
        p.profile_begin()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            p.collide(f, out=q)
        e1.record()
        torch.cuda.synchronize()
        prof = p.profile_end()
        clocks = sampler.stop()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")   # the slowest rank's time
        p.stream_status()
        return ms, prof, clocks

    ms, prof, clocks = timed(plan, a.steps, a.warmup)
    value = job_throughput(world, B, a.steps, ms / 1e3)
    measured = measure_peaks()

    # roofline of the dominant kernel (translate-product), from the library's own events
    per_launch_ms = prof["gain_ms"] / max(1, prof["gain_timed"])
    nodes_per_launch = prof["nodes"] / max(1, prof["gain_launches"])
    flops_node = translate_flops_per_node(N, Nr, npairs, prec)
    achieved = flops_node * nodes_per_launch / (per_launch_ms / 1e3) / 1e12
    peaks = _peaks()
    if prec in ("fp32", "fp64"):
        peak = measured["fp32_fma_tflops"] if prec == "fp32" else measured["fp64_fma_tflops"]
        roof = {"bound": "alu", "peak_source": "measured %s FMA rate of this GPU (of measured)" % prec.upper()}
    else:
        # dense fp16 and bf16 tensor rates are equal; the kernel runs for the whole step
        peak = peaks.get("bf16_tflops_sustained") or 1700.0
        roof = {"bound": "tensor", "peak_source": "MEASURED_PEAKS bf16_tflops_sustained (of measured)"
                if peaks.get("bf16_tflops_sustained") else "fallback 1.7 PFLOP/s sustained"}
    # the method's own work (the translates counted as radix-2 FFTs, Appendix) over the same kernel time
    alg_node = fft_algorithmic_flops_per_node(N, Nr, npairs)
    alg_rate = alg_node * nodes_per_launch / (per_launch_ms / 1e3) / 1e12
    alg_peak = measured["fp32_fma_tflops"] if prec in ("fp32", "fp64") else measured["fp16_dense_tflops"]
    roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                 "frac_basis": "flops the kernel executes (dense circulant passes, split products)"
                 if prec not in ("fp32", "fp64") else "flops of the Fourier-space translates the kernel executes",
                 "achieved_algorithmic": alg_rate, "peak_algorithmic": alg_peak,
                 "frac_algorithmic": alg_rate / alg_peak,
                 "algorithmic_basis": "N_rho (M/2) (5 N^3 log2 N^3 + 20 N^3) per node over the kernel time, against the "
                                      "measured dense %s rate (of measured)" % ("FP32 FMA" if prec in ("fp32", "fp64")
                                                                              else "fp16 cuBLAS"),
                 "traffic": (TRAFFIC_PER_NODE.get((prec, N, Nr, 2 * npairs)) or 0) * nodes_per_launch or None,
                 "traffic_unit": "bytes per launch", "kernel": "translate-product",
                 "kernel_share": prof["gain_ms"] / ms if ms else None,
                 "flops_per_node": flops_node, "nodes_per_launch": nodes_per_launch, "launch_ms": per_launch_ms,
                 **shape_ceiling_fields(N, Nr, npairs, prec, measured, per_launch_ms, nodes_per_launch, clocks),
                 "fft_algorithmic_tflops": fft_algorithmic_flops_per_node(N, Nr, npairs) * value / world / 1e12})

    line = {"metric": METRIC, "value": value, "unit": "node-evals/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[prec],
            "data": "synthetic",
            "config": {"workload": "%s: %d two-Maxwellian nodes/GPU, N=32 on [-7,7]^3, omega=0.74, "
                                   "N_rho=32, M=%d, SVD 1e-8" % (WORKLOAD, B, M),
                       "nodes_per_gpu": B, "N": N, "M": M, "N_rho": Nr,
                       "svd_rank": plan.info["svd_rank_used"], "precision": prec,
                       "chunk_nodes": plan.info["chunk_nodes"],
                       "workspace_gb": round(plan.info["workspace_bytes"] / 2 ** 30, 2),
                       "l2": "no flush: inputs %d MB (%s L2, 129 MB); each chunk writes and re-reads %d MB "
                             "of translate products" % (f.numel() * 4 >> 20,
                                                        "larger than" if f.numel() * 4 > 129 << 20 else "within",
                                                        plan.info["chunk_nodes"] * Nr * N ** 3 * 4 >> 20),
                       "parallelism": "dp%d" % world},
            "gpu_launches": prof["launches"], "clocks": clocks, "roofline": roof, "peaks_measured": measured,
            "tuning": tuning}

    # end to end through the host-buffer entry point (pinned host memory, copies inside)
    if not a.no_e2e:
        fh = torch.from_numpy(F).pin_memory()
        qh = torch.empty_like(fh).pin_memory()
        plan.collide_host(fh, qh)
        barrier()
        t0 = time.perf_counter()
        ke = max(1, a.steps)
        for _ in range(ke):
            plan.collide_host(fh, qh)
        barrier()
        dt = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
        line["e2e"] = {"value": job_throughput(world, B, ke, dt), "unit": "node-evals/s",
                       "h2d_bytes_per_step": fh.numel() * 4, "d2h_bytes_per_step": qh.numel() * 4}

    # the other forms on the same nodes: the plain FP32 GPU form and the other 16-bit mode
    outputs = {prec: q.clone()}
    values = {prec: value}
    if not a.no_compare:
        line["compare"] = {}
        for other in MODES:
            if other == prec:
                continue
            po = binding.Plan(N=N, L=L, gamma=cfg["gamma"], M=M, N_rho=Nr, svd_tol=cfg["svd_tol"], precision=other,
                              max_batch=a.chunk if a.chunk > 0 else B)
            tuning[other] = po.autotune(f)
            ko = max(1, a.steps // 2)
            mso, profo, _ = timed(po, ko, 1)
            outputs[other] = q.clone()
            values[other] = job_throughput(world, B, ko, mso / 1e3)
            line["compare"][other] = {"value": values[other], "unit": "node-evals/s",
                                      "translate_kernel_ms_per_node": profo["gain_ms"] / max(1, profo["nodes"])}
            po.close()
        plan.collide(f, out=q)
        torch.cuda.synchronize()

    # CPU baseline: the oracle on a bounded sample of the same nodes (rank 0, N = 1 only)
    if world == 1 and not a.no_cpu and M == cfg["M"]:   # the oracle sample uses the workload's rule
        plan.collide(f, out=q)
        torch.cuda.synchronize()
        cores = os.cpu_count() or 1
        procs = max(1, min(cores, 16))
        rng = np.random.default_rng(0)
        idx = sorted(rng.choice(B, procs, replace=False).tolist())
        res, comp, wall, used = oracle_sample(idx, B, cfg["seed"], plan.info["svd_rank_used"], procs)
        acc = accuracy_of(outputs, res)
        line["cpu_baseline"] = {"value": len(idx) / comp, "unit": "node-evals/s", "cores": used,
                                "kind": "oracle",
                                "sample": "%d of the %d nodes, one single-threaded FP64 process each" % (len(idx), B)}
        line["accuracy"] = {"vs": "FP64 oracle on the cpu_baseline sample", "nodes": len(idx),
                            "measure": "relative L2 error of the sampled nodes as one vector, by ||Q|| and by the "
                                       "loss term ||Q-||; node_max_* are the largest per-node values", **acc}
        if not a.no_compare:
            line["equal_accuracy"] = equal_accuracy(values, acc)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
