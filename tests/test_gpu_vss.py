"""Parity of the VSS-kernel CUDA path (alpha != 1; eq. B_gen, Appendix eqs. realGG, lowrank1,
apndx_fs_Glm_Qk) with the FP64 oracle, through the C ABI.

Error measure and tolerances as in test_gpu_parity: relative L2 error normalised by the oracle's
loss term, FP64 1e-10, FP32 1e-5. The full-size workload (N = 32, M = 38, N_rho = 32) is checked
through properties that hold at any size: alpha = 2 reproduces the (separately oracle-checked)
VHS path, and Maxwell molecules relax the stress at the closed-form rate of their alpha.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import vss as V
from paper_1809_10186_gb300 import binding, workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1809_10186_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def _dev(a, prec):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float64 if prec == "fp64" else torch.float32)


def _as_input(a, prec):
    return a.astype(np.float64) if prec == "fp64" else a.astype(np.float32).astype(np.float64)


def _err(got, ref, f, g, op):
    loss = f * np.real(op.idft3(op.Gloss * op.dft3(g)))
    return np.linalg.norm(got - ref) / np.linalg.norm(loss)


@pytest.mark.parametrize("prec,N,M,Nrho,loss", [("fp64", 8, 12, 8, "paper"), ("fp64", 16, 26, 8, "conservative"),
                                                ("fp32", 8, 26, 8, "paper"), ("fp32", 16, 12, 16, "paper"),
                                                ("fp64", 12, 12, 6, "paper"), ("fp32", 12, 6, 6, "conservative")])
def test_vss_collide_matches_oracle(prec, N, M, Nrho, loss):
    L, gamma, alpha = 3.5, 0.52, 1.6
    F = _as_input(W.rough(3, N, 300 + N), prec)
    plan = binding.Plan(N=N, L=L, gamma=gamma, alpha=alpha, M=M, N_rho=Nrho, precision=prec, loss=loss)
    assert plan.info["alpha"] == alpha
    q = plan.collide(_dev(F, prec)).double().cpu().numpy()
    plan.stream_status()
    op = V.VSSPlan(N, L, gamma=gamma, alpha=alpha, M=M, Nrho=Nrho, nyquist="sym", loss=loss)
    for i in range(3):
        e = _err(q[i], V.fast_Q_vss(op, F[i]), F[i], F[i], op)
        print(prec, N, M, i, "err/|Q-| %.3g" % e)
        assert e < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_vss_collide2_and_jvp_match_oracle(prec):
    N, L, gamma, alpha, M = 8, 3.0, 0.38, 1.3, 12
    F, G = _as_input(W.rough(2, N, 17), prec), _as_input(W.rough(2, N, 18), prec)
    plan = binding.Plan(N=N, L=L, gamma=gamma, alpha=alpha, M=M, N_rho=6, precision=prec, b=0.07)
    op = V.VSSPlan(N, L, gamma=gamma, alpha=alpha, M=M, Nrho=6, nyquist="sym", b=0.07)
    f, g = _dev(F, prec), _dev(G, prec)
    q2 = plan.collide2(f, g).double().cpu().numpy()
    jv = plan.collide_jvp(f, g).double().cpu().numpy()
    plan.stream_status()
    for i in range(2):
        assert _err(q2[i], V.fast_Q_vss(op, F[i], G[i]), F[i], G[i], op) < TOL[prec]
        ref = V.fast_Q_vss(op, F[i], G[i]) + V.fast_Q_vss(op, G[i], F[i])
        assert _err(jv[i], ref, F[i], G[i], op) < TOL[prec]


def test_vss_n32_reduced_rule_chunked_matches_oracle():
    """N = 32 FP32 with a reduced quadrature (the oracle's table stays small), max_batch = 3 over
    7 nodes: three transform batches with a ragged tail."""
    N, L, gamma, alpha, M, Nrho, B = 32, 7.0, W.omega_to_gamma(0.81), 1.4, 6, 6, 7
    F, _ = W.two_maxwellian(B, N, L, 41, dtype=np.float32)
    F = F.astype(np.float64)
    plan = binding.Plan(N=N, L=L, gamma=gamma, alpha=alpha, M=M, N_rho=Nrho, precision="fp32", max_batch=3)
    q = plan.collide(_dev(F, "fp32")).double().cpu().numpy()
    plan.stream_status()
    op = V.VSSPlan(N, L, gamma=gamma, alpha=alpha, M=M, Nrho=Nrho, nyquist="sym")
    worst = 0.0
    for i in (0, 3, 6):
        worst = max(worst, _err(q[i], V.fast_Q_vss(op, F[i]), F[i], F[i], op))
    print("N=32 VSS FP32 reduced rule worst err/|Q-| %.3g" % worst)
    assert worst < TOL["fp32"]
    assert np.isfinite(q).all()


def test_vss_alpha_two_equals_vhs_at_full_size():
    """alpha = 2 has an isotropic symmetrised kernel with b_vss(omega, 2) = b_vhs(omega): the VSS
    path (608 transforms per node) must reproduce the VHS path on the full workload."""
    cfg = W.CONFIGS["vss_n32"]
    N, L, B = cfg["N"], cfg["L"], cfg["B"]
    F, _ = W.two_maxwellian(B, N, L, cfg["seed"], dtype=np.float32)
    f = _dev(F, "fp32")
    vss = binding.Plan(N=N, L=L, gamma=cfg["gamma"], alpha=2.0, M=cfg["M"], N_rho=cfg["Nrho"], precision="fp32")
    vhs = binding.Plan(N=N, L=L, gamma=cfg["gamma"], M=cfg["M"], N_rho=cfg["Nrho"], precision="fp32")
    a = vss.collide(f)
    b = vhs.collide(f)
    vss.stream_status()
    err = torch.linalg.vector_norm(a - b).item() / torch.linalg.vector_norm(b).item()
    print("alpha = 2 VSS vs VHS at N = 32, %d nodes: rel %.3g" % (B, err))
    assert err < 1e-4


def test_vss_maxwell_molecules_stress_rate_at_full_size():
    """omega = 1: dP_dev/dt = -3 alpha n / (Gamma(3/2)(alpha+1)(alpha+2)) P_dev for any f; checked on
    the N = 32, M = 38, N_rho = 32 grid in FP32 for every node of a batch of bimodal inputs."""
    N, L, alpha, B = 32, 7.0, 1.4, 4
    rng = np.random.default_rng(9)
    c = -L + (np.arange(N) + 0.5) * 2 * L / N
    cx, cy, cz = np.meshgrid(c, c, c, indexing="ij")
    F = np.empty((B, N, N, N))
    for i in range(B):
        ux, T1, T2 = rng.uniform(0.2, 0.5), rng.uniform(0.7, 0.9), rng.uniform(1.1, 1.4)
        F[i] = (0.6 * (np.pi * T1) ** -1.5 * np.exp(-((cx - ux) ** 2 + cy ** 2 + cz ** 2) / T1)
                + 0.4 * (np.pi * T2) ** -1.5 * np.exp(-((cx + 1.5 * ux) ** 2 + cy ** 2 + cz ** 2) / T2))
    plan = binding.Plan(N=N, L=L, gamma=0.0, alpha=alpha, M=38, N_rho=32, precision="fp32")
    F = F.astype(np.float32).astype(np.float64)
    q = plan.collide(_dev(F, "fp32")).double().cpu().numpy()
    plan.stream_status()
    dv = (2 * L / N) ** 3
    for i in range(B):
        n = F[i].sum() * dv
        u = np.array([(F[i] * x).sum() for x in (cx, cy, cz)]) * dv / n
        d = np.stack([cx - u[0], cy - u[1], cz - u[2]])
        P = 2 * np.einsum("aijk,bijk,ijk->ab", d, d, F[i]) * dv
        Pdot = 2 * np.einsum("aijk,bijk,ijk->ab", d, d, q[i]) * dv
        dev = lambda A: A - np.trace(A) / 3 * np.eye(3)
        lam = -(dev(Pdot) * dev(P)).sum() / (dev(P) ** 2).sum()
        closed = V.stress_rate_maxwell(alpha, n)
        print("node %d stress rate %.6f closed form %.6f" % (i, lam, closed))
        assert lam == pytest.approx(closed, rel=3e-3)


def test_vss_ssprk_matches_oracle():
    N, L, alpha, M = 8, 3.5, 1.5, 12
    F = _as_input(W.two_maxwellian(2, N, L, 23)[0], "fp64")
    plan = binding.Plan(N=N, L=L, gamma=0.3, alpha=alpha, M=M, N_rho=8, precision="fp64")
    f = _dev(F, "fp64")
    plan.ssprk(f, 0.05, 3, order=3)
    plan.stream_status()
    op = V.VSSPlan(N, L, gamma=0.3, alpha=alpha, M=M, Nrho=8, nyquist="sym")
    for i in range(2):
        ref = F[i].copy()
        for _ in range(3):
            v1 = ref + 0.05 * V.fast_Q_vss(op, ref)
            v2 = 0.75 * ref + 0.25 * v1 + 0.25 * 0.05 * V.fast_Q_vss(op, v1)
            ref = ref / 3 + 2 / 3 * v2 + 2 / 3 * 0.05 * V.fast_Q_vss(op, v2)
        got = f[i].cpu().numpy()
        assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_vss_unsupported_calls_are_rejected():
    plan = binding.Plan(N=8, L=3.0, alpha=1.5, M=6, N_rho=4, precision="fp64")
    f = torch.rand(2, 8, 8, 8, dtype=torch.float64, device="cuda")
    for call in (lambda: plan.collide_vjp(f, f), lambda: plan.collide_dgamma(f), lambda: plan.collide_noalloc(f)):
        with pytest.raises(binding.DGFSError) as ex:
            call()
        assert "UNSUPPORTED" in str(ex.value)
    with pytest.raises(binding.DGFSError):
        binding.Plan(N=16, L=3.0, alpha=1.5, M=6, precision="f16s")
    with pytest.raises(binding.DGFSError):
        binding.Plan(N=8, L=3.0, alpha=1.5, M=6, svd_tol=1e-6)
    with pytest.raises(binding.DGFSError):
        binding.RaggedSchedule([plan], [0], [0])
    # the plan still works after the rejected calls
    q = plan.collide(f)
    plan.stream_status()
    assert torch.isfinite(q).all()


def test_vss_empty_batch_and_single_node():
    plan = binding.Plan(N=8, L=3.0, alpha=1.7, M=6, N_rho=4, precision="fp64")
    empty = torch.empty(0, 8, 8, 8, dtype=torch.float64, device="cuda")
    assert plan.collide(empty).shape == (0, 8, 8, 8)
    F = _as_input(W.rough(1, 8, 71), "fp64")
    q = plan.collide(_dev(F, "fp64")).cpu().numpy()
    plan.stream_status()
    op = V.VSSPlan(8, 3.0, gamma=0.0, alpha=1.7, M=6, Nrho=4, nyquist="sym")
    assert _err(q[0], V.fast_Q_vss(op, F[0]), F[0], F[0], op) < TOL["fp64"]
