"""Host arithmetic of bench.py (no GPU): the flop counts and MMA-shape ceilings behind the bench
line's roofline fields, and its accuracy and equal-accuracy bookkeeping. Each is checked against an
independent count (pass by pass, MMA by MMA) or a constructed case whose answer is known."""
import importlib.util
import math
import os

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _dense_translate_flops(N, products):
    """Two translates per (radial point, pair), each three 1-D circulant passes: N^2 lines of an
    N x N matrix-vector product (2 N flops per output), every product done once per filter part."""
    flops = 0
    for _translate in range(2):
        for _axis in range(3):
            flops += N * N * N * (2 * N) * products
    return flops


@pytest.mark.parametrize("prec,products", [("f16s", 2), ("bf16s", 2), ("f16x3", 3), ("bf16x3", 3)])
def test_executed_flops_count_every_dense_pass(bench, prec, products):
    N, Nrho, npairs = 32, 32, 19
    per_step = _dense_translate_flops(N, products) + 3 * N ** 3   # + product and weighted sum
    assert bench.translate_flops_per_node(N, Nrho, npairs, prec) == Nrho * npairs * per_step


def test_executed_flops_at_the_headline_workload(bench):
    # the figure the bench line prints as roofline.flops_per_node for F16S at N = 32, M = 38
    assert bench.translate_flops_per_node(32, 32, 19, "f16s") == 15360589824


def test_fourier_space_flops_use_the_radix2_count(bench):
    # a complex radix-2 FFT of n points takes 5 n log2 n flops; the 3-D transform has n = N^3
    N, Nrho, npairs = 16, 16, 3
    n = N ** 3
    fft = 5 * n * math.log2(n)
    assert bench.translate_flops_per_node(N, Nrho, npairs, "fp32") == pytest.approx(Nrho * npairs * (fft + 17 * n))
    assert bench.fft_algorithmic_flops_per_node(N, Nrho, npairs) == pytest.approx(Nrho * npairs * (fft + 20 * n))
    assert bench.fft_algorithmic_flops_per_node(32, 32, 19) == pytest.approx(1892679680.0)


def _mma_table():
    # distinct values so that a wrong shape or operand source shows in the sum
    return {"smem_n32": 41.0, "smem_n64": 47.0, "smem_n128": 67.0, "smem_n256": 131.0,
            "tmem_n64": 79.0, "tmem_n128": 83.0, "tmem_n256": 137.0}


def test_mma_shape_ceiling_counts_the_kernels_mmas(bench):
    mma = _mma_table()
    N = 32
    T, ks = N * N // 128, N // 16          # 128-row tiles, K = 16 steps
    # F16S: pass 1 hi and lo per K step (N = 2n, A in TMEM); passes 2 and 3 one MMA per sign and
    # K step (N = 2n, A in shared memory)
    p1 = sum(mma["tmem_n64"] for _t in range(T) for _k in range(ks) for _part in ("hi", "lo"))
    p23 = sum(mma["smem_n64"] for _p in (2, 3) for _t in range(T) for _s in "+-" for _k in range(ks))
    assert bench.mma_shape_ceiling(N, "f16s", mma) == (pytest.approx(p1 + p23), 1)
    assert bench.mma_shape_ceiling(N, "bf16s", mma) == (pytest.approx(p1 + p23), 1)
    # split data: a CTA pair per step, half the tiles each; pass 1 one N = 4n and one N = 2n MMA
    # per K step, passes 2 and 3 one N = 2n and one N = n MMA per sign and K step
    th = T // 2
    x1 = sum(mma["tmem_n128"] + mma["tmem_n64"] for _t in range(th) for _k in range(ks))
    x23 = sum(mma["smem_n64"] + mma["smem_n32"] for _p in (2, 3) for _t in range(th) for _s in "+-"
              for _k in range(ks))
    assert bench.mma_shape_ceiling(N, "f16x3", mma) == (pytest.approx(x1 + x23), 2)
    # no ceiling for the CUDA-core precisions or a shape the probe did not time
    assert bench.mma_shape_ceiling(N, "fp32", mma) == (None, None)
    assert bench.mma_shape_ceiling(16, "f16s", mma) == (None, None)   # tmem_n32 was not timed


def test_shape_ceiling_fields_convert_launch_time_to_cycles_per_step(bench):
    mma = _mma_table()
    ceil, _ = bench.mma_shape_ceiling(32, "f16s", mma)
    measured = {"mma_cycles": mma, "sms": 152}
    # 152 nodes x 2 radial points x 3 pairs on 152 SMs at 1000 MHz: a 0.06 ms launch is
    # 60000 cycles per SM over 6 steps per SM, i.e. 10000 cycles per step
    f = bench.shape_ceiling_fields(32, 2, 3, "f16s", measured, 0.06, 152, {"sm_mhz": 1000.0})
    assert f["kernel_cycles_per_step"] == pytest.approx(10000.0)
    assert f["mma_shape_cycles_per_step"] == pytest.approx(ceil)
    assert f["frac_of_mma_shape_ceiling"] == pytest.approx(ceil / 10000.0)
    # the split-data kernel spends two CTAs on every step
    ceil3, _ = bench.mma_shape_ceiling(32, "f16x3", mma)
    f3 = bench.shape_ceiling_fields(32, 2, 3, "f16x3", measured, 0.06, 152, {"sm_mhz": 1000.0})
    assert f3["kernel_cycles_per_step"] == pytest.approx(5000.0)
    assert f3["frac_of_mma_shape_ceiling"] == pytest.approx(ceil3 / 5000.0)
    # the maximum clock stands in when no sample was taken; nothing without any clock
    g = bench.shape_ceiling_fields(32, 2, 3, "f16s", measured, 0.06, 152, {"sm_max_mhz": 2000.0})
    assert g["kernel_cycles_per_step"] == pytest.approx(20000.0)
    assert bench.shape_ceiling_fields(32, 2, 3, "f16s", measured, 0.06, 152, {}) == {}
    assert bench.shape_ceiling_fields(32, 2, 3, "fp32", measured, 0.06, 152, {"sm_mhz": 1000.0}) == {}


def _oracle_sample(rng, B, n):
    """[(node, Q, loss)] with zero-sum Q (a conserving operator) and a loss term 20 times larger."""
    res = []
    for i in range(B):
        q = rng.standard_normal(n)
        q -= q.mean()
        res.append((i, q, 20.0 * rng.standard_normal(n)))
    return res


def test_accuracy_of_a_uniformly_scaled_result(bench):
    rng = np.random.default_rng(3)
    B, n, eps = 3, 64, 4e-4
    res = _oracle_sample(rng, B, n)
    Q = np.stack([q for _, q, _ in res])
    got = torch.from_numpy(Q * (1.0 + eps))
    a = bench.accuracy_of({"f16s": got}, res)["f16s"]
    # every node is off by eps ||Q_i||: eps by ||Q|| (batch and per node), eps ||Q|| / ||Q-|| by the loss
    nq = np.sqrt(sum(float(q @ q) for _, q, _ in res))
    nl = np.sqrt(sum(float(l @ l) for _, _, l in res))
    assert a["rel_l2_vs_Q"] == pytest.approx(eps, rel=1e-9)
    assert a["node_max_vs_Q"] == pytest.approx(eps, rel=1e-9)
    assert a["rel_l2_vs_loss"] == pytest.approx(eps * nq / nl, rel=1e-9)
    assert a["mass_drift_max"] < 1e-14                 # the scaled result still sums to zero
    assert a["meets_tolerance"] and a["tolerance_vs_Q"] == bench.TOL_Q["f16s"]
    # 5 eps misses F16S's 1e-3 of ||Q|| though it stays within the loss tolerance
    b = bench.accuracy_of({"f16s": torch.from_numpy(Q * (1.0 + 5 * eps))}, res)["f16s"]
    assert b["rel_l2_vs_Q"] > bench.TOL_Q["f16s"] > b["rel_l2_vs_loss"]
    assert not b["meets_tolerance"]


def test_accuracy_of_reports_mass_drift_and_the_worst_node(bench):
    rng = np.random.default_rng(5)
    res = _oracle_sample(rng, 2, 32)
    Q = np.stack([q for _, q, _ in res])
    got = Q.copy()
    got[1] += 1e-3                                     # node 1 gains 32e-3 of mass
    a = bench.accuracy_of({"fp32": torch.from_numpy(got)}, res)["fp32"]
    _, q1, l1 = res[1]
    assert a["mass_drift_max"] == pytest.approx(32e-3 / np.abs(l1).sum(), rel=1e-9)
    assert a["node_max_vs_Q"] == pytest.approx(np.sqrt(32) * 1e-3 / np.linalg.norm(q1), rel=1e-9)
    assert not a["meets_tolerance"]


def _acc(q, l):
    return {"rel_l2_vs_Q": q, "rel_l2_vs_loss": l}


def test_equal_accuracy_compares_only_modes_within_each_level(bench):
    values = {"fp32": 10.0, "f16s": 40.0, "bf16s": 41.0, "f16x3": 17.0}
    acc = {"fp32": _acc(9e-6, 5e-7), "f16s": _acc(8e-4, 5e-5), "bf16s": _acc(7e-3, 4e-4),
           "f16x3": _acc(7e-6, 4e-7)}
    out = bench.equal_accuracy(values, acc)
    assert set(out["1e-05"]["modes"]) == {"fp32", "f16x3"}
    assert out["1e-05"]["fastest"] == "f16x3"
    assert out["1e-05"]["fastest_over_fp32"] == pytest.approx(1.7)
    # BF16S is the fastest mode overall but outside 1e-3 of ||Q||, so it is in neither level
    assert set(out["0.001"]["modes"]) == {"fp32", "f16s", "f16x3"}
    assert out["0.001"]["fastest"] == "f16s"
    assert out["0.001"]["fastest_over_fp32"] == pytest.approx(4.0)
    # both normalisations must be within the level
    out2 = bench.equal_accuracy({"fp32": 10.0, "f16s": 40.0}, {"fp32": _acc(2e-5, 1e-6), "f16s": _acc(9e-4, 2e-3)})
    assert "1e-05" not in out2
    assert out2["0.001"]["modes"] == {"fp32": 10.0}
    # no FP32 among the qualifying modes: no ratio
    out3 = bench.equal_accuracy({"f16x3": 17.0}, {"f16x3": _acc(7e-6, 4e-7)})
    assert "fastest_over_fp32" not in out3["1e-05"]
