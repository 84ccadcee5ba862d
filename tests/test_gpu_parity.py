"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Error measure: the relative L2 error of a batch, ||Q_gpu - Q_oracle|| / ||Q_oracle|| with all
checked nodes taken as one vector, and the same error normalised by the oracle's loss term ||Q-||
(the magnitude of what the kernels add up: gain and loss cancel to ||Q|| = 0.7-14 % of ||Q-|| on
the two-Maxwellian workloads). Both are asserted against the tolerance of the precision; the
largest per-node values of both are printed. Per node, ||Q||-normalised FP32 errors cannot reach
1e-5 at the nodes nearest equilibrium: an FP32 Fourier stage alone (exact translates) gives
4.7e-5 there (tests/test_precision_floor.py), so the per-node figure is reported, not asserted.

Tolerances (batch, by ||Q|| and by ||Q-||): FP64 1e-10; FP32 1e-5. The modes with 16-bit data
operands round the three stored intermediates of every translate to 11 (fp16) or 8 (bf16)
significand bits: F16S reaches 7e-4 by ||Q|| on the N = 32 workload but 4e-3 on coarse N = 16
grids, BF16S 7e-3 and 3e-2; their tolerances are 1e-2 / 5e-2 by ||Q|| and 1e-3 / 5e-3 by ||Q-||
(the bilinear calls, polarised into two quadratic evaluations, double the bf16 rounding),
and neither meets the 1e-3 of the BF16-split tolerance everywhere: the split-data modes do.
F16X3 (fp16 hi + lo on data and filters, three products, FP32 accumulation) is held to the FP32
tolerance 1e-5, BF16X3 to 1e-3 by ||Q|| and 1e-4 by ||Q-||.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_1809_10186_gb300 import binding, workloads as W

from oracle_refs import batch_errors, references, sample_nodes

pytestmark = pytest.mark.gpu

TOL_Q = {"fp64": 1e-10, "fp32": 1e-5, "f16s": 1e-2, "bf16s": 5e-2, "f16x3": 1e-5, "bf16x3": 1e-3}
TOL_L = {"fp64": 1e-10, "fp32": 1e-5, "f16s": 1e-3, "bf16s": 5e-3, "f16x3": 1e-5, "bf16x3": 1e-4}
TC_PRECS = ("f16s", "bf16s", "f16x3", "bf16x3")
TOL = TOL_L


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1809_10186_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def _dev(a, prec):
    prec = "fp32" if prec in TC_PRECS else prec
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float64 if prec == "fp64" else torch.float32)


def _as_input(a, prec):
    """The values both sides see: rounded to the GPU element type, then FP64 for the oracle."""
    prec = "fp32" if prec in TC_PRECS else prec
    return a.astype(np.float64) if prec == "fp64" else a.astype(np.float32).astype(np.float64)


def _errors(got, ref, loss):
    d = np.linalg.norm(got - ref)
    return d / np.linalg.norm(loss), d / np.linalg.norm(ref)


def _check(prec, got, ref, loss, label, tol_q=None, tol_l=None):
    """Assert the batch errors of Q (lists of per-node arrays) by ||Q|| and by ||Q-||."""
    e = batch_errors(got, ref, loss)
    print("%s %s: batch err/|Q| %.3g err/|Q-| %.3g; worst node err/|Q| %.3g err/|Q-| %.3g" % (
        label, prec, e["batch_q"], e["batch_loss"], e["node_q"], e["node_loss"]))
    assert e["batch_q"] < (tol_q or TOL_Q[prec]), e
    assert e["batch_loss"] < (tol_l or TOL_L[prec]), e
    return e


def _oplan(N, L, gamma, M, Nrho, **kw):
    return O.OraclePlan(N, L, gamma=gamma, M=M, Nrho=Nrho, nyquist="sym", **kw)


# ---- small grids, rough inputs: every entry point ------------------------------------------

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("N", [8, 12, 16, 24])
def test_collide_rough_small(prec, N):
    """Every grid size of the Fourier-space translates (radix-2 lines for 8, 16; one radix-3 stage
    for 12, 24) against the oracle on rough inputs (all modes populated)."""
    L, gamma, M = 3.0, 0.52, 12
    Nr = N if N <= 16 else 8
    F = _as_input(W.rough(3, N, 100 + N), prec)
    plan = binding.Plan(N=N, L=L, gamma=gamma, M=M, N_rho=Nr, precision=prec)
    q = plan.collide(_dev(F, prec)).double().cpu().numpy()
    plan.stream_status()
    op = _oplan(N, L, gamma, M, Nr)
    refs = [O.fast_Q(op, F[i]) for i in range(3)]
    _check(prec, list(q), refs, [np.real(O.loss_Q(op, F[i], F[i])) for i in range(3)], "rough N=%d" % N)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_collide2_jvp_dgamma_small(prec):
    N, L, gamma, M = 8, 3.0, 0.38, 26
    F, G = _as_input(W.rough(2, N, 7), prec), _as_input(W.rough(2, N, 8), prec)
    plan = binding.Plan(N=N, L=L, gamma=gamma, M=M, N_rho=6, precision=prec, b=0.07)
    op = O.OraclePlan(N, L, gamma=gamma, M=M, Nrho=6, nyquist="sym", b=0.07)
    f, g = _dev(F, prec), _dev(G, prec)
    q2 = plan.collide2(f, g).double().cpu().numpy()
    jv = plan.collide_jvp(f, g).double().cpu().numpy()
    dg = plan.collide_dgamma(f).double().cpu().numpy()
    plan.stream_status()
    loss = [np.real(O.loss_Q(op, F[i], G[i])) for i in range(2)]
    _check(prec, list(q2), [O.fast_Q(op, F[i], G[i]) for i in range(2)], loss, "Q(f,g)")
    jloss = [np.real(O.loss_Q(op, F[i], G[i]) + O.loss_Q(op, G[i], F[i])) for i in range(2)]
    _check(prec, list(jv), [O.jvp(op, F[i], G[i]) for i in range(2)], jloss, "JVP")
    dop = O.dgamma_plan(op)
    _check(prec, list(dg), [O.dQ_dgamma(op, F[i]) for i in range(2)],
           [np.real(O.loss_Q(dop, F[i], F[i])) for i in range(2)], "dQ/dgamma")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_vjp_small(prec):
    N, L, gamma, M = 8, 3.0, 0.52, 12
    F, U = _as_input(W.rough(2, N, 17), prec), _as_input(W.rough(2, N, 18) - 0.5, prec)
    plan = binding.Plan(N=N, L=L, gamma=gamma, M=M, N_rho=6, precision=prec)
    op = O.OraclePlan(N, L, gamma=gamma, M=M, Nrho=6, nyquist="sym")
    gf = plan.collide_vjp(_dev(F, prec), _dev(U, prec)).double().cpu().numpy()
    plan.stream_status()
    e = batch_errors(list(gf), [O.vjp(op, F[i], U[i]) for i in range(2)])
    print("VJP", prec, e)
    assert e["batch_q"] < TOL_Q[prec]


@pytest.mark.parametrize("prec", TC_PRECS)
def test_tensor_core_plans_bilinear_and_adjoint_calls(prec):
    """Tensor-core plans run Q(f, f), dQ/dgamma and, by polarisation of the symmetric translate-product
    sum (two quadratic launches on f + a g and f - a g), Q(f, g) and the JVP on the tensor cores: the
    plan's accuracy there; the VJP runs through the FP32 Fourier-space translates: FP32 accuracy."""
    N, L, gamma, M = 16, 5.0, 0.38, 12
    F, G = _as_input(W.rough(2, N, 27), "fp32"), _as_input(W.rough(2, N, 28) - 0.5, "fp32")
    plan = binding.Plan(N=N, L=L, gamma=gamma, M=M, N_rho=8, precision=prec)
    op = O.OraclePlan(N, L, gamma=gamma, M=M, Nrho=8, nyquist="sym")
    f, g = _dev(F, "fp32"), _dev(G, "fp32")
    q2 = plan.collide2(f, g).double().cpu().numpy()
    jv = plan.collide_jvp(f, g).double().cpu().numpy()
    gf = plan.collide_vjp(f, g).double().cpu().numpy()
    qq = plan.collide(f).double().cpu().numpy()
    plan.stream_status()
    loss = [np.real(O.loss_Q(op, F[i], G[i])) for i in range(2)]
    _check(prec, list(q2), [O.fast_Q(op, F[i], G[i]) for i in range(2)], loss, "Q(f,g), tensor cores")
    jloss = [np.real(O.loss_Q(op, F[i], G[i]) + O.loss_Q(op, G[i], F[i])) for i in range(2)]
    _check(prec, list(jv), [O.jvp(op, F[i], G[i]) for i in range(2)], jloss, "JVP, tensor cores")
    e = batch_errors(list(gf), [O.vjp(op, F[i], G[i]) for i in range(2)])
    assert e["batch_q"] < TOL_Q["fp32"], e
    _check(prec, list(qq), [O.fast_Q(op, F[i]) for i in range(2)],
           [np.real(O.loss_Q(op, F[i], F[i])) for i in range(2)], "Q(f,f)")


@pytest.mark.parametrize("prec", ["f16x3", "bf16x3", "f16s"])
def test_tensor_core_jvp_n32_sampled(prec):
    """The differentiation workload's JVP (512 nodes, N = 32, M = 38, unit-norm Gaussian directions) on
    the tensor cores by polarisation, against the oracle on 16 nodes; F16X3 at the FP32 tolerance."""
    cfg = W.CONFIGS["grad_n32"]
    N, L, B = cfg["N"], cfg["L"], cfg["B"]
    F, _ = W.two_maxwellian(B, N, L, cfg["seed"], dtype=np.float32)
    V = W.directions(B, N, cfg["seed"] + 100, dtype=np.float32)
    plan = binding.Plan(N=N, L=L, gamma=cfg["gamma"], M=cfg["M"], N_rho=cfg["Nrho"], precision=prec)
    jv = plan.collide_jvp(_dev(F, "fp32"), _dev(V, "fp32")).double().cpu().numpy()
    plan.stream_status()
    idx = sample_nodes(B, 16)
    refs = references("grad", "grad_n32", idx)
    e = batch_errors([jv[i] for i in idx], [refs[i]["jvp"] for i in idx], [refs[i]["jvp_loss"] for i in idx])
    print("N=32 JVP %s on %d nodes: %s" % (prec, len(idx), e))
    assert e["batch_q"] < TOL_Q[prec] and e["batch_loss"] < TOL_L[prec], e


# ---- the workload configurations -------------------------------------------------------------

@pytest.mark.parametrize("N", [16, 24, 32])
def test_bkw_error_table_on_the_gpu_fp64(N, golden_dir):
    """The paper's BKW table (FP64, its Titan-X runs) reproduced by the FP64 GPU path: every entry
    for this N within a factor 1.5 (|Q - Q_exact|_inf; domain [-6.62, 6.62]^3, B = 1/(4 pi),
    the paper's M = 6 half-sphere design = our 12-point rule)."""
    import os
    rows = []
    with open(os.path.join(golden_dir, "bkw_table1.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                v = line.split()
                if int(v[0]) == N:
                    rows.append((int(v[1]), [float(x) for x in v[2:5]]))
    L = 6.62
    c = -L + (np.arange(N) + 0.5) * 2 * L / N
    cx, cy, cz = np.meshgrid(c, c, c, indexing="ij")
    c2 = cx * cx + cy * cy + cz * cz
    for nr, errs in rows:
        plan = binding.Plan(N=N, L=L, gamma=0.0, b=1.0 / (4.0 * math.pi), M=12, N_rho=nr, precision="fp64")
        F = np.stack([O.bkw_f(c2, t0) for t0 in (5.5, 6.5, 10.0)])
        q = plan.collide(_dev(F, "fp64")).cpu().numpy()
        plan.stream_status()
        for i, (t0, ref) in enumerate(zip((5.5, 6.5, 10.0), errs)):
            err = np.abs(q[i] - O.bkw_Q(c2, t0)).max()
            print("N=%d N_r=%d t0=%g GPU err %.3g paper %.3g" % (N, nr, t0, err, ref))
            assert ref / 1.5 < err < ref * 1.5
        plan.close()


def test_bkw_single_node_fp64():
    """Single node, Maxwell molecules, BKW datum at t0 = 5.5, N = 16, FP64; with the stated
    R = 2 sqrt2 L / (3 + sqrt2) and with the paper's default R; 20 SSP-RK2 steps of 0.01."""
    cfg = W.CONFIGS["bkw_n16"]
    N, L = cfg["N"], cfg["L"]
    f0 = W.bkw(N, L, 5.5)
    for R in (cfg["R"], O.default_R(L)):
        plan = binding.Plan(N=N, L=L, gamma=0.0, b=cfg["b"], R=R, M=cfg["M"], N_rho=cfg["Nrho"], precision="fp64")
        op = O.OraclePlan(N, L, gamma=0.0, b=cfg["b"], R=R, M=cfg["M"], Nrho=cfg["Nrho"], nyquist="sym")
        q = plan.collide(_dev(f0[None], "fp64")).cpu().numpy()[0]
        ref = O.fast_Q(op, f0)
        e_loss, e_q = _errors(q, ref, np.real(O.loss_Q(op, f0, f0)))
        c2 = O.grid_c2(op)
        print("R=%.4f err/|Q-| %.3g err/|Q| %.3g  |Q-Q_bkw|_inf %.3g" % (R, e_loss, e_q, np.abs(q - O.bkw_Q(c2, 5.5)).max()))
        assert e_q < 1e-10
        # 20 SSP-RK2 steps (eq. SSPRK2) by the library's own stepper (dgfs_ssprk)
        f = _dev(f0[None], "fp64")
        plan.ssprk(f, 0.01, 20, order=2)
        plan.stream_status()
        fo = O.ssp_rk2(op, f0, 0.01, 20)
        assert np.abs(f.cpu().numpy()[0] - fo).max() < 1e-13
        print("  after 20 steps |f - f_bkw(5.7)|_inf = %.3g" % np.abs(fo - O.bkw_f(c2, 5.7)).max())
    # direct O(N^6) sum at N = 8 against the device result (paper lattice == sym here: smooth)
    plan8 = binding.Plan(N=8, L=L, gamma=0.0, b=cfg["b"], M=cfg["M"], N_rho=8, precision="fp64")
    f8 = W.bkw(8, L, 5.5)
    op8 = O.OraclePlan(8, L, gamma=0.0, b=cfg["b"], M=cfg["M"], Nrho=8, nyquist="paper")
    q8 = plan8.collide(_dev(f8[None], "fp64")).cpu().numpy()[0]
    d8 = O.direct_Q(op8, f8)
    assert np.linalg.norm(q8 - d8) / np.linalg.norm(d8) < 1e-8


@pytest.mark.parametrize("prec,order", [("fp64", 2), ("fp64", 3), ("fp32", 3)])
def test_ssprk_matches_oracle_and_follows_bkw(prec, order):
    """dgfs_ssprk (eqs. SSPRK2, SSPRK3) on a batch of BKW data against the oracle's schemes, with
    a scale factor (1/Kn) and more nodes than one internal chunk."""
    cfg = W.CONFIGS["bkw_n16"]
    N, L = cfg["N"], cfg["L"]
    f0 = W.bkw(N, L, 5.5)
    plan = binding.Plan(N=N, L=L, gamma=0.0, b=cfg["b"], R=cfg["R"], M=cfg["M"], N_rho=cfg["Nrho"], precision=prec,
                        max_batch=2)
    op = O.OraclePlan(N, L, gamma=0.0, b=cfg["b"], R=cfg["R"], M=cfg["M"], Nrho=cfg["Nrho"], nyquist="sym")
    scale, dt, steps = 0.5, 0.02, 10      # df/dt = 0.5 Q: the BKW datum at t0 + 0.5 * 0.2
    F0 = np.stack([f0] * 3)
    f = _dev(_as_input(F0, prec), prec)
    plan.ssprk(f, dt, steps, order=order, scale=scale)
    plan.stream_status()
    scheme = O.ssp_rk2 if order == 2 else O.ssp_rk3
    ref = scheme(op, _as_input(f0, prec), dt * scale, steps)   # scale folds into the step
    got = f.double().cpu().numpy()
    err = np.abs(got - ref[None]).max() / np.abs(ref).max()
    print(prec, "RK%d" % order, "rel max err vs oracle %.3g, |f - f_bkw|_inf %.3g" % (
        err, np.abs(ref - O.bkw_f(O.grid_c2(op), 5.6)).max()))
    assert err < (1e-12 if prec == "fp64" else 1e-6)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_moments_and_entropy_match_oracle(prec):
    N, L = 16, 6.0
    F, _ = W.two_maxwellian(4, N, L, 808)
    F = _as_input(F, prec)
    plan = binding.Plan(N=N, L=L, gamma=0.38, M=12, N_rho=N, precision=prec)
    mom = plan.moments(_dev(F, prec)).cpu().numpy()
    op = O.OraclePlan(N, L, gamma=0.38, M=12, Nrho=N, nyquist="sym")
    tol = 1e-12 if prec == "fp64" else 1e-6
    for i in range(4):
        m = O.moments(op, F[i])
        ref = [m["n"], *m["u"], m["T"], m["P"][0, 0], m["P"][1, 1], m["P"][2, 2], m["P"][0, 1], m["P"][0, 2],
               m["P"][1, 2], *m["q"], O.entropy(op, F[i])]
        np.testing.assert_allclose(mom[i], ref, rtol=tol, atol=tol * max(1.0, abs(m["n"])))


def test_entropy_decreases_along_device_steps():
    """H-theorem along dgfs_ssprk: a two-Maxwellian mixture relaxes, H decreases, mass, momentum
    and energy stay (loss in the paper's form conserves them to the spectral error)."""
    N, L = 16, 6.0
    F, _ = W.two_maxwellian(2, N, L, 909)
    plan = binding.Plan(N=N, L=L, gamma=0.38, M=12, N_rho=N, precision="fp64")
    f = _dev(F, "fp64")
    hist = [plan.moments(f).cpu().numpy()]
    for _ in range(4):
        plan.ssprk(f, 0.05, 2, order=3)
        hist.append(plan.moments(f).cpu().numpy())
    plan.stream_status()
    H = np.array([h[:, 14] for h in hist])
    assert (np.diff(H, axis=0) < 0).all(), H
    n = np.array([h[:, 0] for h in hist])
    assert np.abs(n / n[0] - 1).max() < 1e-3


def test_slab_n24_fp32_all_nodes():
    cfg = W.CONFIGS["slab_n24"]
    N, L, B = cfg["N"], cfg["L"], cfg["B"]
    F, _ = W.two_maxwellian(B, N, L, cfg["seed"])
    F = _as_input(F, "fp32")
    plan = binding.Plan(N=N, L=L, gamma=cfg["gamma"], M=cfg["M"], N_rho=cfg["Nrho"], precision="fp32")
    q = plan.collide(_dev(F, "fp32")).double().cpu().numpy()
    plan.stream_status()
    op = _oplan(N, L, cfg["gamma"], cfg["M"], cfg["Nrho"])
    _check("fp32", list(q), [O.fast_Q(op, F[i]) for i in range(B)],
           [np.real(O.loss_Q(op, F[i], F[i])) for i in range(B)], "slab N=24, all %d nodes" % B)


N32_NODES = 24   # nodes of the 2048-node launch checked against the oracle


# the primary workload's stated tolerance of the split 16-bit forms (1e-3 relative, by ||Q||), which
# F16S meets there although coarse grids need its general 1e-2
PRIMARY_TOL_Q = {"f16s": 1e-3}


def _vhs32(cfg_name, prec, nodes_checked=N32_NODES):
    """The whole 2048-node launch on the device; batch errors on `nodes_checked` sampled nodes."""
    cfg = W.CONFIGS[cfg_name]
    N, L, B = cfg["N"], cfg["L"], cfg["B"]
    F, _ = W.two_maxwellian(B, N, L, cfg["seed"], dtype=np.float32)
    plan = binding.Plan(N=N, L=L, gamma=cfg["gamma"], M=cfg["M"], N_rho=cfg["Nrho"],
                        svd_tol=cfg.get("svd_tol", 0.0), precision=prec)
    q = plan.collide(_dev(F, prec)).double().cpu().numpy()
    plan.stream_status()
    assert np.isfinite(q).all()
    idx = sample_nodes(B, nodes_checked)
    refs = references("Q", cfg_name, idx, plan.info["svd_rank_used"] if cfg.get("svd_tol") else 0)
    e = _check(prec, [q[i] for i in idx], [refs[i]["Q"] for i in idx], [refs[i]["loss"] for i in idx],
               "N=32 %d-node launch, %d nodes checked (rank %d)" % (B, len(idx), plan.info["svd_rank_used"]),
               tol_q=PRIMARY_TOL_Q.get(prec) if cfg_name == "vhs_n32" else None)
    return e, plan


def test_vhs_n32_full_batch_fp32_sampled():
    """The primary workload's launch (2048 nodes, N = 32, M = 38, SVD at 1e-8) in FP32."""
    _vhs32("vhs_n32", "fp32")


def test_derivatives_n32_fp32():
    cfg = W.CONFIGS["grad_n32"]
    N, L, B = cfg["N"], cfg["L"], cfg["B"]
    F, _ = W.two_maxwellian(B, N, L, cfg["seed"], dtype=np.float32)
    V = W.directions(B, N, cfg["seed"] + 100, dtype=np.float32)
    U = W.directions(B, N, cfg["seed"] + 200, dtype=np.float32)
    plan = binding.Plan(N=N, L=L, gamma=cfg["gamma"], M=cfg["M"], N_rho=cfg["Nrho"], precision="fp32")
    f, v, u = _dev(F, "fp32"), _dev(V, "fp32"), _dev(U, "fp32")
    jv = plan.collide_jvp(f, v).double().cpu().numpy()
    gf = plan.collide_vjp(f, u).double().cpu().numpy()
    dg = plan.collide_dgamma(f).double().cpu().numpy()
    plan.stream_status()
    idx = sample_nodes(B, 16)
    refs = references("grad", "grad_n32", idx)
    for name, got, lossname in (("jvp", jv, "jvp_loss"), ("vjp", gf, None), ("dgamma", dg, "dgamma_loss")):
        e = batch_errors([got[i] for i in idx], [refs[i][name] for i in idx],
                         [refs[i][lossname] for i in idx] if lossname else None)
        print("N=32 FP32 %s on %d nodes: %s" % (name, len(idx), e))
        assert e["batch_q"] < TOL_Q["fp32"], (name, e)
        if lossname:
            assert e["batch_loss"] < TOL_L["fp32"], (name, e)
    # dot-product identity on the device results, every checked node
    for i in idx:
        lhs, rhs = float(np.dot(U[i].ravel(), jv[i].ravel())), float(np.dot(gf[i].ravel(), V[i].ravel()))
        assert abs(lhs - rhs) < 1e-5 * abs(lhs), (i, lhs, rhs)


def test_jvp_central_difference_fp64():
    """JVP against central differences of the device Q (exact: Q is quadratic)."""
    N, L = 16, 5.0
    F, _ = W.two_maxwellian(2, N, L, 3)
    V = W.directions(2, N, 4)
    plan = binding.Plan(N=N, L=L, gamma=0.38, M=12, N_rho=N, precision="fp64")
    f, v = _dev(F, "fp64"), _dev(V, "fp64")
    h = 1e-3
    fd = (plan.collide(f + h * v) - plan.collide(f - h * v)) / (2 * h)
    jv = plan.collide_jvp(f, v)
    assert (torch.linalg.norm(jv - fd) / torch.linalg.norm(jv)).item() < 1e-9
    # dgamma against central differences in gamma (b held fixed)
    b = plan.info["b"]
    pp = binding.Plan(N=N, L=L, gamma=0.38 + 1e-4, b=b, M=12, N_rho=N, precision="fp64")
    pm = binding.Plan(N=N, L=L, gamma=0.38 - 1e-4, b=b, M=12, N_rho=N, precision="fp64")
    fdg = (pp.collide(f) - pm.collide(f)) / 2e-4
    dg = plan.collide_dgamma(f)
    assert (torch.linalg.norm(dg - fdg) / torch.linalg.norm(dg)).item() < 1e-6


def test_ragged_mixed_grids():
    """Packed nodes of N = 16, 24, 32 with per-node omega, in one call."""
    cfg = W.CONFIGS["cavity_ragged"]
    B = 60
    node_N, node_omega = W.ragged_layout(B, cfg["Ns"], cfg["split"], cfg["omegas"], cfg["seed"])
    L, M = cfg["L"], cfg["M"]
    plans = {n: binding.Plan(N=n, L=L, M=M, N_rho=n, precision="fp32") for n in cfg["Ns"]}
    order = list(cfg["Ns"])
    offs = np.zeros(B, np.int64)
    tot = 0
    for i in range(B):
        offs[i] = tot
        tot += int(node_N[i]) ** 3
    packed = np.zeros(tot, np.float32)
    fields = []
    for i in range(B):
        n = int(node_N[i])
        fi = W.near_equilibrium(1, n, L, cfg["seed"] + i, dtype=np.float32)[0]
        fields.append(fi)
        packed[offs[i]:offs[i] + n ** 3] = fi.ravel()
    gam = 2 * (1 - node_omega)
    bb = np.array([O.b_vhs(w) for w in node_omega])
    fp = torch.from_numpy(packed).cuda()
    q = binding.collide_ragged([plans[n] for n in order], [order.index(int(n)) for n in node_N], offs, fp,
                               node_gamma=gam, node_b=bb).cpu().numpy()
    for p in plans.values():
        p.stream_status()
    worst = 0
    for i in list(range(0, B, 7)) + [B - 1]:
        n = int(node_N[i])
        op = _oplan(n, L, gam[i], M, n, b=bb[i])
        Fi = fields[i].astype(np.float64)
        e, _ = _errors(q[offs[i]:offs[i] + n ** 3].reshape(n, n, n), O.fast_Q(op, Fi), np.real(O.loss_Q(op, Fi, Fi)))
        worst = max(worst, e)
    print("ragged worst err/|Q-| %.3g" % worst)
    assert worst < TOL["fp32"]


def _ragged_case(B, Ns, split, seed, L):
    omegas = (0.5, 0.74, 0.81)
    node_N, node_omega = W.ragged_layout(B, Ns, split, omegas, seed)
    offs = np.zeros(B, np.int64)
    tot = 0
    for i in range(B):
        offs[i] = tot
        tot += int(node_N[i]) ** 3
    packed = np.zeros(tot, np.float32)
    for i in range(B):
        n = int(node_N[i])
        packed[offs[i]:offs[i] + n ** 3] = W.near_equilibrium(1, n, L, seed + i, dtype=np.float32)[0].ravel()
    gam = 2 * (1 - node_omega)
    bb = np.array([O.b_vhs(w) for w in node_omega])
    return node_N, offs, packed, gam, bb


@pytest.mark.parametrize("prec,Ns", [("fp32", (16, 24, 32)), ("f16s", (16, 24, 32)), ("f16x3", (16, 24, 32))])
def test_ragged_schedule_equals_call_and_replays_in_a_graph(prec, Ns):
    """dgfs_ragged_create/collide: device-resident layout, identical to dgfs_collide_ragged, and a
    CUDA-graph capture of a whole mixed-N batch replays to the same result on new inputs."""
    L, M, B = 9.0, 26, 40
    split = tuple([1.0 / len(Ns)] * len(Ns))
    node_N, offs, packed, gam, bb = _ragged_case(B, Ns, split, 4242, L)
    plans = [binding.Plan(N=n, L=L, M=M, N_rho=n, precision=prec) for n in Ns]
    cls = [list(Ns).index(int(n)) for n in node_N]
    fp = torch.from_numpy(packed).cuda()
    ref = binding.collide_ragged(plans, cls, offs, fp, node_gamma=gam, node_b=bb)
    sched = binding.RaggedSchedule(plans, cls, offs, node_gamma=gam, node_b=bb)
    q = sched.collide(fp)
    torch.cuda.synchronize()
    for p in plans:
        p.stream_status()
    assert torch.equal(q, ref)
    # capture the whole mixed-N batch once, replay on another input
    x = fp.clone()
    y = torch.empty_like(fp)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        sched.collide(x, out=y, stream=s)   # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sched.collide(x, out=y, stream=s)
    _, _, packed2, _, _ = _ragged_case(B, Ns, split, 777, L)
    x.copy_(torch.from_numpy(packed2).cuda())
    g.replay()
    torch.cuda.synchronize()
    direct = sched.collide(torch.from_numpy(packed2).cuda())
    torch.cuda.synchronize()
    for p in plans:
        p.stream_status()
    assert torch.equal(y, direct)
    sched.close()


# ---- structural properties and the C ABI's contract ----------------------------------------------

def test_chunking_batch_order_and_determinism():
    N, L = 16, 5.0
    F, _ = W.two_maxwellian(7, N, L, 11, dtype=np.float32)
    f = _dev(F, "fp32")
    p1 = binding.Plan(N=N, L=L, gamma=0.38, M=12, N_rho=N, precision="fp32")
    p3 = binding.Plan(N=N, L=L, gamma=0.38, M=12, N_rho=N, precision="fp32", max_batch=3)
    assert p3.info["chunk_nodes"] == 3
    a = p1.collide(f)
    assert torch.equal(a, p1.collide(f))                     # bitwise reproducible
    assert torch.equal(a, p3.collide(f))                     # chunking does not change results
    perm = torch.tensor([3, 0, 6, 1, 5, 2, 4], device="cuda")
    assert torch.equal(a[perm], p1.collide(f[perm].contiguous()))


@pytest.mark.parametrize("prec,N", [("fp64", 8), ("fp32", 16), ("f16s", 32), ("f16s", 24), ("bf16s", 16),
                                    ("f16x3", 32), ("f16x3", 24), ("bf16x3", 16)])
def test_zero_field_sign_and_scale_invariants(prec, N):
    """Degenerate and scaled inputs in one batch with ordinary nodes: a zero field gives exactly zero
    (no NaN flag: the 16-bit forms' per-node scale falls back to 1), Q is even (Q(-f) equals Q(f)
    bitwise: negation commutes with every rounding, the 16-bit scale is taken from |f|) and
    homogeneous of degree 2 (Q(2^k f) = 4^k Q(f): power-of-two factors are exact in every form, the
    16-bit data being rescaled per node, so only values that cross the FP32 subnormal range differ)."""
    L = {8: 3.0, 16: 5.0, 24: 6.0, 32: 7.0}[N]
    F, _ = W.two_maxwellian(2, N, L, 91, dtype=np.float32)
    F = F.astype(np.float32)
    zero = np.zeros((1, N, N, N), np.float32)
    batch = np.concatenate([zero, F, -F, F * np.float32(2.0 ** -8), F * np.float32(2.0 ** 8)])
    plan = binding.Plan(N=N, L=L, gamma=0.52, M=12, N_rho=8, precision=prec)
    q = plan.collide(_dev(batch, prec)).double().cpu()
    plan.stream_status()   # raises on a NaN / infinity flag
    assert torch.isfinite(q).all()
    assert torch.equal(q[0], torch.zeros_like(q[0]))
    base = q[1:3]
    assert torch.equal(q[3:5], base)
    for i, k in ((5, -8), (7, 8)):
        scaled = q[i:i + 2] * 4.0 ** (-k)
        rel = (torch.linalg.norm((scaled - base).flatten()) / torch.linalg.norm(base.flatten())).item()
        assert rel < 1e-6, (prec, N, k, rel)
    plan.close()


@pytest.mark.parametrize("max_batch,B,pinned", [(1, 3, True), (2, 5, True), (7, 5, False), (0, 9, True),
                                                (4, 37, True), (64, 300, True), (0, 2, True)])
def test_host_buffer_entry_point_matches_device(max_batch, B, pinned):
    """The host-buffer call pipelines its copies over sub-batches (one staging buffer when the
    plan's chunk is one node, two otherwise; sizes ramping up from B / 32 and down at the end,
    the middle ones up to half the chunk); every node's result equals the device call's, on two consecutive
    calls (the second reuses the staging buffers while the first's are fresh)."""
    N, L = 16, 5.0
    plan = binding.Plan(N=N, L=L, gamma=0.38, M=12, N_rho=N, precision="fp32", max_batch=max_batch)
    for call in range(2):
        F, _ = W.two_maxwellian(B, N, L, 12 + call, dtype=np.float32)
        fh = torch.from_numpy(F)
        qh = torch.empty_like(fh)
        if pinned:
            fh, qh = fh.pin_memory(), qh.pin_memory()
        plan.collide_host(fh, qh)
        assert torch.equal(qh, plan.collide(fh.cuda()).cpu()), (max_batch, B, call)
    plan.close()


def test_empty_batch_and_argument_errors():
    plan = binding.Plan(N=8, L=3.0, gamma=0.0, M=6, N_rho=4, precision="fp32")
    f = torch.rand(2, 8, 8, 8, device="cuda")
    out = torch.empty_like(f)
    L_ = binding.lib()
    s = binding._stream_ptr()
    import ctypes
    assert L_.dgfs_collide(plan.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()), 0, s) == 0
    # misaligned pointer
    assert L_.dgfs_collide(plan.handle, ctypes.c_void_p(f.data_ptr() + 4), ctypes.c_void_p(out.data_ptr()), 1, s) == 1
    # output aliasing the input
    assert L_.dgfs_collide(plan.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(f.data_ptr()), 1, s) == 1
    # negative batch
    assert L_.dgfs_collide(plan.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()), -1, s) == 1
    with pytest.raises(binding.DGFSError):                       # FP64 VSS is limited to N <= 24
        binding.Plan(N=32, L=7.0, M=38, alpha=1.4, precision="fp64")


def test_autograd_function():
    N, L = 8, 3.0
    plan = binding.Plan(N=N, L=L, gamma=0.52, M=12, N_rho=6, precision="fp64")
    F = W.rough(1, N, 3)
    f = _dev(F, "fp64").requires_grad_(True)
    q = binding.collide(plan, f)
    u = torch.randn_like(q)
    (g,) = torch.autograd.grad(q, f, u)
    op = O.OraclePlan(N, L, gamma=0.52, M=12, Nrho=6, nyquist="sym")
    ref = O.vjp(op, F[0], u[0].cpu().numpy())
    assert np.linalg.norm(g[0].cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-10


def test_autograd_gamma_gradient():
    """gamma as a differentiable input of binding.collide: reverse mode with a scalar gamma and with
    one gamma per node, and forward mode, against the oracle's dQ/dgamma contracted with the upstream
    gradient and against central differences of the device Q in gamma (b held fixed), FP64."""
    N, L, g0, M = 16, 5.0, 0.38, 12
    plan = binding.Plan(N=N, L=L, gamma=g0, M=M, N_rho=N, precision="fp64")
    b = plan.info["b"]
    F, _ = W.two_maxwellian(2, N, L, 31)
    Ug = W.directions(2, N, 32)
    u = _dev(Ug, "fp64")
    op = O.OraclePlan(N, L, gamma=g0, b=b, M=M, Nrho=N, nyquist="sym")
    per_node = np.array([np.sum(Ug[i] * O.dQ_dgamma(op, F[i])) for i in range(2)])
    # scalar gamma, together with the gradient of f
    f = _dev(F, "fp64").requires_grad_(True)
    gam = torch.tensor(g0, dtype=torch.float64, device="cuda", requires_grad=True)
    gg, gf = torch.autograd.grad((binding.collide(plan, f, gam) * u).sum(), (gam, f))
    assert abs(gg.item() - per_node.sum()) < 1e-10 * abs(per_node.sum())
    assert np.linalg.norm(gf[0].cpu().numpy() - O.vjp(op, F[0], Ug[0])) < 1e-10 * np.linalg.norm(gf[0].cpu().numpy())
    # central differences of the device Q in gamma
    h = 1e-4
    pp = binding.Plan(N=N, L=L, gamma=g0 + h, b=b, M=M, N_rho=N, precision="fp64")
    pm = binding.Plan(N=N, L=L, gamma=g0 - h, b=b, M=M, N_rho=N, precision="fp64")
    fd = (((pp.collide(f.detach()) - pm.collide(f.detach())) * u).sum() / (2 * h)).item()
    assert abs(gg.item() - fd) < 1e-6 * abs(fd)
    # one gamma per node
    gvec = torch.full((2,), g0, dtype=torch.float64, device="cuda", requires_grad=True)
    (gv,) = torch.autograd.grad((binding.collide(plan, f, gvec) * u).sum(), (gvec,))
    np.testing.assert_allclose(gv.cpu().numpy(), per_node, rtol=1e-10)
    # forward mode: tangent of Q along gamma_dot = 1 is dQ/dgamma
    import torch.autograd.forward_ad as fwAD
    with fwAD.dual_level():
        gd = fwAD.make_dual(gam.detach(), torch.ones((), dtype=torch.float64, device="cuda"))
        qd = binding.collide(plan, f.detach(), gd)
        tangent = fwAD.unpack_dual(qd).tangent
    for i in range(2):
        ref = O.dQ_dgamma(op, F[i])
        assert np.linalg.norm(tangent[i].cpu().numpy() - ref) < 1e-10 * np.linalg.norm(ref)
    # a gamma that differs from the plan's is refused
    with pytest.raises(ValueError):
        binding.collide(plan, f, torch.tensor(g0 + 0.1, dtype=torch.float64, device="cuda"))


# ---- tensor-core (tcgen05) translates ---------------------------------------------------------

@pytest.mark.parametrize("prec", TC_PRECS)
@pytest.mark.parametrize("N,kind", [(16, "rough"), (16, "smooth"), (32, "smooth"), (32, "rough")])
def test_tensor_core_collide(prec, N, kind):
    L, gamma, M = (3.0 if kind == "rough" else 6.0), 0.52, 12
    F = W.rough(3, N, 300 + N) if kind == "rough" else W.two_maxwellian(3, N, L, 301 + N)[0]
    F = _as_input(F, "fp32")
    plan = binding.Plan(N=N, L=L, gamma=gamma, M=M, N_rho=N, precision=prec)
    q = plan.collide(_dev(F, "fp32")).double().cpu().numpy()
    plan.stream_status()
    op = _oplan(N, L, gamma, M, N)
    _check(prec, list(q), [O.fast_Q(op, F[i]) for i in range(3)],
           [np.real(O.loss_Q(op, F[i], F[i])) for i in range(3)], "tensor cores N=%d %s" % (N, kind))


@pytest.mark.parametrize("prec", TC_PRECS)
@pytest.mark.parametrize("kind", ["smooth", "rough"])
def test_tensor_core_n24_on_padded_tiles(prec, kind):
    """N = 24 (the radix-3 grid) on the 32-point tensor-core tiles: zero-padded filters and data give the
    24-point translate products exactly (the kernels read and write only the 24^3 block), against the
    oracle at the precision's tolerances (the split-data precisions at FP32's)."""
    N, L, gamma, M, Nr = 24, (3.0 if kind == "rough" else 6.0), 0.38, 12, 12
    F = W.rough(3, N, 324) if kind == "rough" else W.two_maxwellian(3, N, L, 325)[0]
    F = _as_input(F, "fp32")
    plan = binding.Plan(N=N, L=L, gamma=gamma, M=M, N_rho=Nr, precision=prec)
    q = plan.collide(_dev(F, "fp32")).double().cpu().numpy()
    plan.stream_status()
    op = _oplan(N, L, gamma, M, Nr)
    _check(prec, list(q), [O.fast_Q(op, F[i]) for i in range(3)],
           [np.real(O.loss_Q(op, F[i], F[i])) for i in range(3)], "tensor cores N=24 %s" % kind)
    # every work-item size gives the same P (items of 1, 2, 3, 4, 6 of the 12 radial points)
    ref = plan.collide(_dev(F, "fp32")).clone()
    for rpc in (1, 2, 3, 4, 6):
        plan.set_tuning(rpc, 0)
        assert torch.equal(plan.collide(_dev(F, "fp32")), ref), rpc
    plan.close()


@pytest.mark.parametrize("prec", ["f16s", "f16x3"])
@pytest.mark.parametrize("N,rule", [(16, 6), (16, 26), (16, 38), (32, 6), (32, "one_pair"), (32, "two_pairs")])
def test_tensor_core_sphere_rules(prec, N, rule):
    """1, 2, 3, 13 and 19 antipodal pairs through the tensor-core kernel (the filter double buffer
    with one or both halves in use and with refills; the rings' phase counts per pair at both
    grid sizes), and rotated user rules with no zero components, against the oracle with the
    same rule."""
    L, gamma = 6.0, 0.52
    if isinstance(rule, int):
        kw, okw = {"M": rule}, {"M": rule}
    else:
        rng = np.random.default_rng(7)
        n = 1 if rule == "one_pair" else 2
        v = rng.normal(size=(n, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        w = np.full(n, 2.0 * np.pi / n)   # weight of each point; the full sphere sums to 4 pi
        kw = {"sphere": np.column_stack([v, w])}
        okw = {"sphere": (np.concatenate([v, -v]), np.concatenate([w, w]))}
    F = _as_input(W.two_maxwellian(2, N, L, 900 + N)[0], "fp32")
    plan = binding.Plan(N=N, L=L, gamma=gamma, N_rho=N, precision=prec, **kw)
    q = plan.collide(_dev(F, "fp32")).double().cpu().numpy()
    plan.stream_status()
    op = O.OraclePlan(N, L, gamma=gamma, Nrho=N, nyquist="sym", **okw)
    assert plan.info["n_pairs"] == len(op.sigma)
    _check(prec, list(q), [O.fast_Q(op, F[i]) for i in range(2)],
           [np.real(O.loss_Q(op, F[i], F[i])) for i in range(2)], "N=%d rule %s" % (N, rule))
    plan.close()


@pytest.mark.parametrize("prec", TC_PRECS)
def test_tensor_core_vhs_n32_full_batch_sampled(prec):
    """The primary workload's launch (2048 nodes, N = 32, M = 38, SVD 1e-8) on tensor cores."""
    _vhs32("vhs_n32", prec)


@pytest.mark.parametrize("prec", ["f16s", "f16x3"])
def test_tensor_core_chunking_and_determinism(prec):
    N, L = 32, 7.0
    F, _ = W.two_maxwellian(5, N, L, 13, dtype=np.float32)
    f = _dev(F, "fp32")
    p1 = binding.Plan(N=N, L=L, gamma=0.52, M=38, N_rho=N, precision=prec)
    p2 = binding.Plan(N=N, L=L, gamma=0.52, M=38, N_rho=N, precision=prec, max_batch=2)
    a = p1.collide(f)
    assert torch.equal(a, p1.collide(f))
    assert torch.equal(a, p2.collide(f))


@pytest.mark.parametrize("prec,rule,B", [("f16s", 6, 200), ("f16s", 38, 200), ("bf16s", 38, 200),
                                         ("f16s", "one_pair", 200), ("f16s", 38, 400), ("f16s", "one_pair", 400),
                                         ("f16x3", 38, 100), ("f16x3", "one_pair", 200), ("bf16x3", 38, 200)])
def test_tensor_core_radial_points_per_cta_equal_one(prec, rule, B):
    """Batches that fill the GPU many times over run several radial points per CTA (one set-up for
    all: the pair sequence continues into the next radial point's filters): two at 200 nodes of
    N_rho = 32, four at 400; small chunks run one radial point per CTA. The schedules perform the
    same arithmetic per radial point, so the results are identical, including for a single sphere
    pair (two or four steps per CTA)."""
    N, L = 32, 7.0
    if isinstance(rule, int):
        kw = {"M": rule}
    else:
        kw = {"sphere": np.array([[0.36, 0.48, 0.8, 2.0 * np.pi]])}
    F, _ = W.two_maxwellian(B, N, L, 91, dtype=np.float32)
    f = _dev(F, "fp32")
    big = binding.Plan(N=N, L=L, gamma=0.52, N_rho=N, precision=prec, max_batch=B, **kw)   # 3200 CTAs of 2 or 4
    small = binding.Plan(N=N, L=L, gamma=0.52, N_rho=N, precision=prec, max_batch=8, **kw)  # 256 CTAs of 1
    a, b = big.collide(f), small.collide(f)
    big.stream_status()
    small.stream_status()
    assert torch.equal(a, b)
    big.close()
    small.close()


@pytest.mark.parametrize("prec", ["f16s", "f16x3"])
def test_lost_hand_off_times_out_and_the_plan_recovers(prec):
    """Failure detection without a GPU fault: the first CTA of the tensor-core kernel withholds
    one hand-off signal (host-injected), its bounded waits give up, the CTA drains and frees its
    resources, the call reports DGFS_ERR_TIMEOUT through dgfs_stream_status, and the next call
    on the same plan returns the normal result."""
    import time
    N, L = 32, 7.0
    F, _ = W.two_maxwellian(3, N, L, 55, dtype=np.float32)
    f = _dev(F, "fp32")
    plan = binding.Plan(N=N, L=L, gamma=0.52, M=6, N_rho=N, precision=prec)
    ref = plan.collide(f)
    plan.stream_status()
    plan.debug_inject(1)
    t0 = time.time()
    plan.collide(f)
    with pytest.raises(binding.DGFSError) as err:
        plan.stream_status()
    print("injected lost signal: %s after %.2f s" % (err.value, time.time() - t0))
    assert "TIMEOUT" in str(err.value)
    again = plan.collide(f)
    plan.stream_status()
    assert torch.equal(again, ref)
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "f16s", "f16x3"])
def test_cuda_graph_capture_equals_eager(prec):
    """dgfs_collide enqueues kernels only, so a captured call replays to the eager result."""
    N, L = 32, 7.0
    F, _ = W.two_maxwellian(3, N, L, 77, dtype=np.float32)
    plan = binding.Plan(N=N, L=L, gamma=0.52, M=12, N_rho=N, precision=prec)
    f = _dev(F, "fp32")
    eager = plan.collide(f)
    q = torch.empty_like(f)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.collide(f, out=q)                      # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.collide(f, out=q)
    q.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(q, eager)
