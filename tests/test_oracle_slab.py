"""Pins of the 1-D DGFS oracle (Sec. 3.1 eqs. eq_weakForm, eq_numericalFlux_upwind, eq_stiffMatrix1;
the diffuse wall condition of Sec. 3.6) against closed forms and structural properties:

  * S: its K = 2 closed form and S + S^T = e_K e_K^T - e_1 e_1^T (integration by parts);
  * DG with the upwind flux is exact for continuous polynomials of degree K - 1 (interior elements);
  * the upwind flux reads the upstream neighbour only;
  * a uniform Maxwellian between walls at its own temperature is stationary under transport;
  * n_w reproduces a wall Maxwellian, and the diffuse walls keep the total mass exactly
    (with the mass-conserving collision loss);
  * a spatially uniform f collides as Q(f, f) / Kn at interior nodes (H sums to M).
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import slab as SL
from oracle.dg import dg_tensors


def _grid(plan):
    return np.meshgrid(plan.c, plan.c, plan.c, indexing="ij")


def _maxw(plan, n, u, T):
    cx, cy, cz = _grid(plan)
    return n * (np.pi * T) ** -1.5 * np.exp(-((cx - u[0]) ** 2 + (cy - u[1]) ** 2 + (cz - u[2]) ** 2) / T)


def test_stiffness_closed_forms():
    np.testing.assert_allclose(SL.stiffness(2), [[-0.5, -0.5], [0.5, 0.5]], atol=1e-15)
    for K in (2, 3, 4, 5):
        S = SL.stiffness(K)
        E = np.zeros((K, K))
        E[0, 0], E[-1, -1] = -1.0, 1.0
        np.testing.assert_allclose(S + S.T, E, atol=1e-13)
        np.testing.assert_allclose(S.sum(axis=0), 0.0, atol=1e-13)    # the derivative of sum_m phi_m = 1


@pytest.mark.parametrize("K", [2, 3, 4])
def test_upwind_dg_is_exact_for_continuous_polynomials(K):
    plan = O.OraclePlan(8, 4.0, M=6, Nrho=4, nyquist="sym")
    edges = np.array([0.0, 0.13, 0.3, 0.52, 0.75, 1.0])
    sl = SL.SlabOracle(plan, K, edges, math.inf, (0, 0, 0, 1.0), (0, 0, 0, 1.0))
    cx, cy, cz = _grid(plan)
    g = np.exp(-(cx ** 2 + cy ** 2 + cz ** 2))
    coef = [1.0, 0.3, -0.5, 0.2][:K]
    xs = sl.node_positions()
    F = np.array([[np.polyval(coef[::-1], x) * g for x in xs[i]] for i in range(sl.I)])
    dcoef = np.polyder(np.array(coef[::-1]))
    exact = np.array([[-cx * np.polyval(dcoef, x) * g for x in xs[i]] for i in range(sl.I)])
    r = sl.rhs(F)
    assert np.abs(r[1:-1] - exact[1:-1]).max() < 1e-12 * np.abs(exact).max()


def test_upwind_flux_reads_the_upstream_neighbour_only():
    plan = O.OraclePlan(8, 4.0, M=6, Nrho=4, nyquist="sym")
    sl = SL.SlabOracle(plan, 3, np.linspace(0, 1, 5), math.inf, (0, 0, 0, 1.0), (0, 0, 0, 1.0))
    rng = np.random.default_rng(3)
    F = rng.random((4, 3, 8, 8, 8))
    r0 = sl.rhs(F)
    cx = sl.c1
    G = F.copy()
    G[2] += np.where(cx > 0, 1.0, 0.0) * rng.random((3, 8, 8, 8))      # downstream of element 1 for c_x > 0
    r1 = sl.rhs(G)
    assert np.abs((r1[1] - r0[1])[:, cx > 0]).max() == 0.0
    assert np.abs((r1[3] - r0[3])[:, cx > 0]).max() > 0.0               # element 3 is downstream of 2
    G = F.copy()
    G[0] += np.where(cx < 0, 1.0, 0.0) * rng.random((3, 8, 8, 8))      # upstream of nothing for c_x < 0
    r2 = sl.rhs(G)
    assert np.abs((r2[1] - r0[1])[:, cx < 0]).max() == 0.0


def test_uniform_maxwellian_between_walls_at_its_temperature_is_stationary():
    plan = O.OraclePlan(8, 4.0, M=6, Nrho=4, nyquist="sym")
    sl = SL.SlabOracle(plan, 3, np.linspace(0, 1, 6), math.inf, (0, 0.0, 0, 0.9), (0, 0.0, 0, 0.9))
    F = np.array([[_maxw(plan, 0.8, (0, 0, 0), 0.9)] * 3] * 5)
    assert np.abs(sl.rhs(F)).max() < 1e-12 * np.abs(F).max()   # round-off of (2/h) M^-1 c_1 S F


def test_wall_density_and_exact_mass_conservation():
    plan = O.OraclePlan(8, 4.0, gamma=0.3, M=12, Nrho=6, nyquist="sym", loss="conservative")
    sl = SL.SlabOracle(plan, 3, [0.0, 0.2, 0.45, 0.7, 1.0], 0.5, (0, 0.2, 0, 0.9), (0, -0.1, 0.05, 1.2))
    fw = SL.wall_maxwellian(plan, (0, 0.2, 0), 0.9)
    assert sl.wall_density(0, 1.7 * fw) == pytest.approx(1.7, rel=1e-14)
    rng = np.random.default_rng(4)
    base = _maxw(plan, 1.0, (0.1, 0.0, 0.0), 1.0)
    F = np.array([[base * (1 + 0.2 * rng.standard_normal(base.shape)) for _ in range(3)] for _ in range(4)])
    r = sl.rhs(F)
    assert abs(sl.mass(r)) < 1e-13 * sl.mass(F)


def test_uniform_state_collides_as_Q_over_Kn():
    plan = O.OraclePlan(8, 4.0, gamma=0.3, M=12, Nrho=6, nyquist="sym")
    f = _maxw(plan, 1.0, (0.3, 0, 0), 0.8) + 0.5 * _maxw(plan, 0.5, (-0.4, 0.2, 0), 1.3)
    Kn = 0.7
    sl = SL.SlabOracle(plan, 3, np.linspace(0, 1, 4), Kn, (0, 0, 0, 1.0), (0, 0, 0, 1.0))
    F = np.array([[f] * 3] * 3)
    r = sl.rhs(F)
    q = O.fast_Q(plan, f) / Kn
    for m in range(3):
        np.testing.assert_allclose(r[1][m], q, atol=1e-12 * np.abs(q).max())


def test_mass_matrix_weights_integrate_the_basis():
    _, M, _ = dg_tensors(3)
    np.testing.assert_allclose(M.sum(axis=0), [1 / 3, 4 / 3, 1 / 3], atol=1e-15)   # Simpson's weights on [-1, 1]
