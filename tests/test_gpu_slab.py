"""Parity of the 1-D DGFS solver on the device (dgfs_slab_*: eq. eq_weakForm with the upwind flux,
diffuse walls, the element collision term and SSP-RK) with the FP64 oracle, through the C ABI.
Errors are relative L2 against the oracle's right-hand side: FP64 1e-10, FP32 1e-5."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import slab as SL
from oracle import vss as V
from paper_1809_10186_gb300 import binding

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1809_10186_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def _maxw(plan, n, u, T):
    cx, cy, cz = np.meshgrid(plan.c, plan.c, plan.c, indexing="ij")
    return n * (np.pi * T) ** -1.5 * np.exp(-((cx - u[0]) ** 2 + (cy - u[1]) ** 2 + (cz - u[2]) ** 2) / T)


def _state(plan, I, K, seed, prec):
    rng = np.random.default_rng(seed)
    F = np.empty((I, K) + (plan.N,) * 3)
    for i in range(I):
        for l in range(K):
            F[i, l] = (_maxw(plan, rng.uniform(0.8, 1.2), (rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), 0),
                             rng.uniform(0.8, 1.2)) * (1 + 0.05 * rng.standard_normal((plan.N,) * 3)))
    return F if prec == "fp64" else F.astype(np.float32).astype(np.float64)


def _dev(a, prec):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float64 if prec == "fp64" else torch.float32)


@pytest.mark.parametrize("prec,K,Kn,loss", [("fp64", 3, 0.5, "paper"), ("fp32", 3, 0.5, "paper"),
                                            ("fp64", 2, math.inf, "paper"), ("fp64", 4, 2.0, "conservative"),
                                            ("fp32", 4, math.inf, "paper")])
def test_slab_rhs_matches_oracle(prec, K, Kn, loss):
    N, L, gamma, M, Nrho = 8, 4.0, 0.38, 12, 6
    edges = [0.0, 0.15, 0.4, 0.7, 1.0]
    wl, wr = (0.0, 0.1, 0.0, 0.9), (0.0, -0.2, 0.05, 1.15)
    plan = binding.Plan(N=N, L=L, gamma=gamma, M=M, N_rho=Nrho, precision=prec, loss=loss)
    slab = binding.Slab(plan, K, edges, Kn, wl, wr)
    op = O.OraclePlan(N, L, gamma=gamma, M=M, Nrho=Nrho, nyquist="sym", loss=loss)
    ref_slab = SL.SlabOracle(op, K, edges, Kn, wl, wr, svd_tol=0.0)
    F = _state(op, len(edges) - 1, K, 11 + K, prec)
    got = slab.rhs(_dev(F, prec)).double().cpu().numpy()
    plan.stream_status()
    ref = ref_slab.rhs(F)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(prec, K, Kn, loss, "rel err %.3g" % err)
    assert err < TOL[prec]
    slab.close()


def test_slab_rhs_with_a_vss_plan():
    N, L, K = 8, 3.5, 3
    edges = np.linspace(0, 1, 4)
    wl, wr = (0.0, 0.0, 0.0, 0.95), (0.0, 0.3, 0.0, 1.05)
    plan = binding.Plan(N=N, L=L, gamma=0.2, alpha=1.5, M=12, N_rho=6, precision="fp64")
    slab = binding.Slab(plan, K, edges, 0.8, wl, wr)
    op = V.VSSPlan(N, L, gamma=0.2, alpha=1.5, M=12, Nrho=6, nyquist="sym")
    F = _state(op, 3, K, 5, "fp64")
    ref = SL.SlabOracle(op, K, edges, 0.8, wl, wr, collide=lambda H, G: sum_direct(op, H, G)).rhs(F)
    got = slab.rhs(_dev(F, "fp64")).cpu().numpy()
    plan.stream_status()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < TOL["fp64"]


def sum_direct(op, H, F):
    """eq. HH with the VSS oracle operator."""
    K = H.shape[0]
    Q = [[V.fast_Q_vss(op, F[a], F[b]) for b in range(K)] for a in range(K)]
    return np.array([sum(H[m, a, b] * Q[a][b] for a in range(K) for b in range(K)) for m in range(K)])


@pytest.mark.parametrize("prec,order", [("fp64", 2), ("fp64", 3), ("fp32", 2)])
def test_slab_ssprk_matches_oracle(prec, order):
    N, L, K, dt, steps = 8, 4.0, 3, 0.004, 3
    edges = np.linspace(0, 1, 5)
    wl, wr = (0.0, 0.0, 0.0, 0.9), (0.0, 0.0, 0.0, 1.1)
    plan = binding.Plan(N=N, L=L, gamma=0.0, M=12, N_rho=6, precision=prec)
    slab = binding.Slab(plan, K, edges, 1.0, wl, wr)
    op = O.OraclePlan(N, L, gamma=0.0, M=12, Nrho=6, nyquist="sym")
    ref_slab = SL.SlabOracle(op, K, edges, 1.0, wl, wr, svd_tol=0.0)
    F = _state(op, 4, K, 21, prec)
    f = _dev(F, prec)
    slab.ssprk(f, dt, steps, order=order)
    plan.stream_status()
    ref = (ref_slab.ssp_rk2 if order == 2 else ref_slab.ssp_rk3)(F, dt, steps)
    err = np.linalg.norm(f.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    print(prec, order, "rel err %.3g" % err)
    assert err < (1e-12 if prec == "fp64" else 1e-6)


def test_slab_conserves_mass_on_the_device():
    """Diffuse walls and the conservative collision loss keep int int f dx dc to round-off."""
    N, L, K = 8, 4.0, 3
    edges = [0.0, 0.1, 0.3, 0.6, 0.85, 1.0]
    wl, wr = (0.0, -0.3, 0.0, 0.8), (0.0, 0.3, 0.0, 1.3)
    plan = binding.Plan(N=N, L=L, gamma=0.5, M=12, N_rho=6, precision="fp64", loss="conservative")
    slab = binding.Slab(plan, K, edges, 0.3, wl, wr)
    op = O.OraclePlan(N, L, gamma=0.5, M=12, Nrho=6, nyquist="sym", loss="conservative")
    ref_slab = SL.SlabOracle(op, K, edges, 0.3, wl, wr)
    F = _state(op, 5, K, 31, "fp64")
    f = _dev(F, "fp64")
    m0 = ref_slab.mass(F)
    slab.ssprk(f, 0.003, 20, order=2)
    plan.stream_status()
    m1 = ref_slab.mass(f.cpu().numpy())
    assert abs(m1 - m0) < 1e-12 * m0


def test_slab_argument_errors():
    plan = binding.Plan(N=8, L=4.0, M=6, N_rho=4, precision="fp64")
    good = dict(K=3, edges=[0.0, 0.5, 1.0], Kn=1.0, wall_left=(0, 0, 0, 1.0), wall_right=(0, 0, 0, 1.0))
    for bad in (dict(K=1), dict(K=9), dict(edges=[0.0, 0.5, 0.5]), dict(Kn=0.0), dict(Kn=-1.0),
                dict(wall_left=(0.1, 0, 0, 1.0)), dict(wall_right=(0, 0, 0, 0.0))):
        kw = dict(good, **bad)
        with pytest.raises(binding.DGFSError):
            binding.Slab(plan, kw["K"], kw["edges"], kw["Kn"], kw["wall_left"], kw["wall_right"])
    slab = binding.Slab(plan, **good)
    F = torch.zeros(2, 3, 8, 8, 8, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.DGFSError):
        slab.rhs(F, out=F)
    with pytest.raises(binding.DGFSError):
        slab.ssprk(F, 0.01, 1, order=4)
    with pytest.raises(binding.DGFSError):
        slab.set_walls((0, 0, 0, 1.0), (0.2, 0, 0, 1.0))
    slab.close()


def test_slab_unsteady_walls_match_oracle():
    """dgfs_slab_set_walls between steps (an oscillating wall): two SSP-RK2 steps at one wall
    velocity, then two at another, against the oracle doing the same."""
    N, L, K, dt = 8, 4.0, 3, 0.004
    edges = np.linspace(0, 1, 4)
    plan = binding.Plan(N=N, L=L, gamma=0.38, M=12, N_rho=6, precision="fp64")
    op = O.OraclePlan(N, L, gamma=0.38, M=12, Nrho=6, nyquist="sym")
    F = _state(op, 3, K, 41, "fp64")
    f = _dev(F, "fp64")
    slab = binding.Slab(plan, K, edges, 0.9, (0, 0.0, 0, 1.0), (0, 0.2, 0, 1.0))
    ref = SL.SlabOracle(op, K, edges, 0.9, (0, 0.0, 0, 1.0), (0, 0.2, 0, 1.0), svd_tol=0.0)
    slab.ssprk(f, dt, 2)
    G = ref.ssp_rk2(F, dt, 2)
    slab.set_walls((0, 0.0, 0, 1.0), (0, -0.3, 0.1, 1.05))
    ref.set_walls((0, 0.0, 0, 1.0), (0, -0.3, 0.1, 1.05))
    slab.ssprk(f, dt, 2)
    plan.stream_status()
    G = ref.ssp_rk2(G, dt, 2)
    assert np.linalg.norm(f.cpu().numpy() - G) / np.linalg.norm(G) < 1e-12


def test_slab_single_element_between_walls():
    """I = 1: both faces of the only element are walls."""
    N, L, K = 8, 4.0, 4
    edges = [0.0, 1.0]
    wl, wr = (0.0, 0.2, 0.0, 0.9), (0.0, -0.1, 0.0, 1.2)
    plan = binding.Plan(N=N, L=L, gamma=0.2, M=12, N_rho=6, precision="fp64")
    slab = binding.Slab(plan, K, edges, 0.6, wl, wr)
    op = O.OraclePlan(N, L, gamma=0.2, M=12, Nrho=6, nyquist="sym")
    F = _state(op, 1, K, 61, "fp64")
    got = slab.rhs(_dev(F, "fp64")).cpu().numpy()
    plan.stream_status()
    ref = SL.SlabOracle(op, K, edges, 0.6, wl, wr, svd_tol=0.0).rhs(F)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < TOL["fp64"]


@pytest.mark.parametrize("prec,order", [("fp64", 3), ("fp32", 2)])
def test_slab_graph_replay_equals_eager_steps(prec, order):
    """Several steps in one call replay a captured step; single-step calls run eagerly. Both give the
    same bits, also after the step size, the plan's tuning and the walls change (each rebuilds the
    graph), and inside a caller's own graph capture (which takes the eager path)."""
    N, L, K = 8, 4.0, 3
    edges = np.linspace(0, 1, 6)
    wl, wr = (0.0, 0.1, 0.0, 0.9), (0.0, -0.2, 0.0, 1.1)
    plan = binding.Plan(N=N, L=L, gamma=0.38, M=12, N_rho=6, precision=prec)
    slab = binding.Slab(plan, K, edges, 0.7, wl, wr)
    op = O.OraclePlan(N, L, gamma=0.38, M=12, Nrho=6, nyquist="sym")
    F = _state(op, 5, K, 51, prec)
    a, b = _dev(F, prec), _dev(F, prec)

    def both(dt, n):
        slab.ssprk(a, dt, n, order=order)
        for _ in range(n):
            slab.ssprk(b, dt, 1, order=order)
        plan.stream_status()
        assert torch.equal(a, b)

    both(0.004, 5)
    both(0.004, 3)
    both(0.002, 4)
    plan.set_tuning(2, 0)
    both(0.002, 2)
    slab.set_walls((0.0, 0.3, 0.0, 1.0), (0.0, 0.0, 0.1, 1.2))
    both(0.002, 3)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        slab.ssprk(a, 0.002, 2, order=order, stream=s)
    g.replay()
    for _ in range(2):
        slab.ssprk(b, 0.002, 1, order=order)
    torch.cuda.synchronize()
    plan.stream_status()
    assert torch.equal(a, b)
    slab.close()
