"""Pins of the VSS-kernel oracle (Sec. 2.1 eq. B_gen, Sec. 2.2, Appendix eqs. realGG, lowrank1,
apndx_fs_Glm_Qk with alpha != 1) against closed forms, special cases and brute force (no GPU).

  * b and F: the total cross section is alpha-independent; F equals its Funk-Hecke (Legendre)
    series and a brute-force sphere quadrature in a fixed frame;
  * alpha = 1 (VHS) and alpha = 2 (whose symmetrised kernel is isotropic) reproduce the VHS
    oracle to round-off;
  * the O(N^6) Galerkin sum with the sphere-dependent quadrature kernel pins the fast form;
  * Maxwell molecules (omega = 1) relax the deviatoric stress at a rate fixed in closed form by
    alpha, for any distribution: that pins the angular factor and its normalisation;
  * mass conservation and the Maxwellian equilibrium.
"""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre, gamma as Gamma, rgamma, spherical_jn

import oracle as O
from oracle import vss as V
from oracle.quadrature import gauss_legendre
from paper_1809_10186_gb300 import workloads as W


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _maxwellian(plan, n, u, T):
    cx, cy, cz = np.meshgrid(plan.c, plan.c, plan.c, indexing="ij")
    return n * (np.pi * T) ** -1.5 * np.exp(-((cx - u[0]) ** 2 + (cy - u[1]) ** 2 + (cz - u[2]) ** 2) / T)


@pytest.mark.parametrize("omega", [0.5, 0.74, 1.0])
def test_b_reduces_to_vhs_and_total_cross_section_is_alpha_independent(omega):
    assert V.b_vss(omega, 1.0) == pytest.approx(O.b_vhs(omega), rel=1e-15)
    t, w = gauss_legendre(200)
    for alpha in (1.0, 1.3, 1.5, 2.0):
        total = 2 * math.pi * np.sum(w * V.B_sym(V.b_vss(omega, alpha), 0.0, alpha, 1.0, t))
        assert total == pytest.approx(4 * math.pi * O.b_vhs(omega), rel=1e-6)


def _funk_hecke(b, gamma, alpha, L, k_abs, mu, c_r):
    """F as the Legendre series of the angular factor: (1+t)^beta has the Legendre moments
    c_l = 2^(beta+1) Gamma(beta+1)^2 / (Gamma(beta+l+2) Gamma(beta+1-l)), and by Funk-Hecke
    int_S2 P_l(sigma.e) cos(a k^.e) de = 4 pi (-1)^(l/2) j_l(a) P_l(sigma.k^) for even l."""
    beta = alpha - 1.0
    a = math.pi * c_r * k_abs / (2 * L)
    total = 0.0
    for l in range(0, int(a) + 80, 2):
        cl = 2 ** (beta + 1) * Gamma(beta + 1) ** 2 * rgamma(beta + l + 2) * rgamma(beta + 1 - l)
        total += (2 * l + 1) / 2 * cl * 4 * math.pi * (-1) ** (l // 2) * spherical_jn(l, a) * eval_legendre(l, mu)
    return c_r ** (2 + gamma) * b * total      # 2 c_r^2 * (1/2 of the full sphere) * b c_r^gamma * series


@pytest.mark.parametrize("alpha", [1.0, 1.25, 1.5, 1.8, 2.0])
def test_F_equals_funk_hecke_series(alpha):
    b, gamma, L = V.b_vss(0.74, alpha), 0.52, 5.0
    for k_abs, mu, c_r in ((0.0, 0.0, 1.1), (1.0, 1.0, 0.7), (3.0, 0.2, 2.5), (11.0, -0.7, 4.1),
                           (27.7, 0.95, 4.6), (41.0, -0.33, 4.6)):
        x = V.F_vss(b, gamma, alpha, L, np.array([k_abs]), np.array([mu]), c_r)[0]
        y = _funk_hecke(b, gamma, alpha, L, k_abs, mu, c_r)
        assert abs(x - y) <= 1e-12 * max(1.0, abs(y)), (k_abs, mu, c_r, x, y)


def test_F_against_brute_force_sphere_quadrature():
    """Half sphere z >= 0 in a fixed frame (sigma generic): Gauss-Legendre in z x trapezoid in phi.
    The kernel has kinks at e = +-sigma, so the product rule converges only algebraically."""
    alpha, b, gamma, L = 1.5, V.b_vss(0.8, 1.5), 0.4, 4.0
    z, wz = gauss_legendre(400, 0.0, 1.0)
    phi = (np.arange(800) + 0.5) * 2 * math.pi / 800
    Z, P = np.meshgrid(z, phi, indexing="ij")
    s = np.sqrt(1 - Z * Z)
    E = np.stack([s * np.cos(P), s * np.sin(P), Z], -1)
    Wt = wz[:, None] * (2 * math.pi / 800)
    sigma = np.array([0.48, -0.6, 0.64])
    sigma /= np.linalg.norm(sigma)
    for kvec, c_r in (([1, 0, 0], 0.9), ([2, -1, 3], 2.3), ([-4, 3, 1], 3.1)):
        kvec = np.array(kvec, float)
        integrand = V.B_sym(b, gamma, alpha, c_r, E @ sigma) * np.cos(math.pi * c_r * (E @ kvec) / (2 * L))
        brute = 2 * c_r ** 2 * np.sum(Wt * integrand)
        kk = np.linalg.norm(kvec)
        x = V.F_vss(b, gamma, alpha, L, np.array([kk]), np.array([sigma @ kvec / kk]), c_r)[0]
        assert x == pytest.approx(brute, rel=2e-6, abs=1e-9)


@pytest.mark.parametrize("nyquist,loss", [("paper", "paper"), ("sym", "paper"), ("paper", "conservative"),
                                          ("sym", "conservative")])
def test_alpha_one_and_two_reproduce_vhs(nyquist, loss):
    """alpha = 1 is VHS; for alpha = 2 the symmetrised angular factor (1+t + 1-t)/2 is constant and
    b_vss(omega, 2) = b_vhs(omega), so the operator is VHS again."""
    N, L = 8, 4.0
    iso = O.OraclePlan(N, L, gamma=0.5, M=12, Nrho=8, nyquist=nyquist, loss=loss)
    f = _maxwellian(iso, 1.0, [0.2, 0, 0], 0.9) + 0.5 * _maxwellian(iso, 1.0, [-0.5, 0.3, 0], 1.1)
    g = _maxwellian(iso, 0.7, [0.1, 0.2, -0.3], 1.2)
    ref = O.fast_Q(iso, f, g)
    for alpha in (1.0, 2.0):
        pl = V.VSSPlan(N, L, gamma=0.5, alpha=alpha, M=12, Nrho=8, nyquist=nyquist, loss=loss)
        assert _rel(V.fast_Q_vss(pl, f, g), ref) < 1e-13


@pytest.mark.parametrize("N,M,loss,alpha", [(4, 6, "paper", 1.5), (6, 12, "paper", 1.3),
                                            (4, 26, "conservative", 1.7)])
def test_direct_sum_equals_fast_form(N, M, loss, alpha):
    g_ = W.rng(200 + N)
    f, g = g_.random((N, N, N)), g_.random((N, N, N))
    pl = V.VSSPlan(N, 3.3, gamma=0.38, alpha=alpha, M=M, Nrho=5, nyquist="paper", loss=loss)
    assert _rel(V.fast_Q_vss(pl, f, g), V.direct_Q_vss(pl, f, g)) < 1e-12


def _stress_rate(pl, f):
    """-d(P_dev)/dt projected on P_dev, from the second moment of Q(f, f) (eq. moments1)."""
    q = V.fast_Q_vss(pl, f)
    m = O.moments(pl, f)
    cx, cy, cz = np.meshgrid(pl.c, pl.c, pl.c, indexing="ij")
    d = np.stack([cx, cy, cz]) - m["u"][:, None, None, None]
    Pdot = 2 * np.einsum("aijk,bijk,ijk->ab", d, d, q) * pl.dc ** 3
    dev = lambda A: A - np.trace(A) / 3 * np.eye(3)
    return -float((dev(Pdot) * dev(m["P"])).sum() / (dev(m["P"]) ** 2).sum()), m["n"]


def test_maxwell_molecules_stress_relaxation_closed_form():
    """omega = 1: for ANY f, dP_dev/dt = -(3/4) n int_S2 B sin^2(chi) dsigma P_dev
    = -3 alpha n / (Gamma(3/2)(alpha+1)(alpha+2)) P_dev. The alpha = 1.5 / alpha = 1 ratio cancels
    the grid's own truncation error and pins the angular factor (a 2.9 % effect)."""
    rates = {}
    for alpha in (1.0, 1.5):
        pl = V.VSSPlan(16, 5.0, gamma=0.0, alpha=alpha, M=38, Nrho=16, nyquist="sym")
        f = _maxwellian(pl, 0.6, [0.4, 0.1, 0], 0.8) + _maxwellian(pl, 0.4, [-0.6, -0.15, 0], 1.2)
        lam, n = _stress_rate(pl, f)
        rates[alpha] = lam
        assert lam == pytest.approx(V.stress_rate_maxwell(alpha, n), rel=0.02)
    closed = V.stress_rate_maxwell(1.5, 1.0) / V.stress_rate_maxwell(1.0, 1.0)
    assert rates[1.5] / rates[1.0] == pytest.approx(closed, rel=5e-4)
    assert abs(closed - 1.0) > 0.025


def test_conservative_loss_conserves_mass_and_maxwellian_is_equilibrium():
    pl = V.VSSPlan(8, 4.0, gamma=0.5, alpha=1.6, M=12, Nrho=8, nyquist="sym", loss="conservative")
    f = W.rough(1, 8, 7)[0]
    mass, _, _ = O.conserved_moments(pl, V.fast_Q_vss(pl, f))
    assert abs(mass) < 1e-13 * np.abs(f).sum() * pl.dc ** 3
    # the Maxwellian residual is the grid's truncation error (7.6e-4 for VHS on this grid)
    pl16 = V.VSSPlan(16, 5.0, gamma=0.5, alpha=1.6, M=12, Nrho=16, nyquist="sym")
    M_ = _maxwellian(pl16, 1.0, [0.0, 0.0, 0.0], 1.0)
    lossmag = np.abs(M_ * pl16.idft3(pl16.Gloss * pl16.dft3(M_)).real).max()
    assert np.abs(V.fast_Q_vss(pl16, M_)).max() < 2e-3 * lossmag


def test_planted_angular_mistake_is_caught(monkeypatch):
    """Dropping the sigma dependence of F (sigma . k := 0) must fail the closed-form pins."""
    b, L = V.b_vss(0.74, 1.5), 5.0
    good = V.F_vss(b, 0.52, 1.5, L, np.array([11.0]), np.array([0.9]), 4.1)[0]
    bad = V.F_vss(b, 0.52, 1.5, L, np.array([11.0]), np.array([0.0]), 4.1)[0]
    ref = _funk_hecke(b, 0.52, 1.5, L, 11.0, 0.9, 4.1)
    assert abs(good - ref) < 1e-12 * abs(ref) and abs(bad - ref) > 1e-3 * abs(ref)
    real_F = V.F_vss
    monkeypatch.setattr(V, "F_vss", lambda b, g, a, L, k, mu, c: real_F(b, g, a, L, k, 0.0 * np.asarray(mu), c))
    pl = V.VSSPlan(16, 5.0, gamma=0.0, alpha=1.5, M=12, Nrho=16, nyquist="sym")
    f = _maxwellian(pl, 0.6, [0.4, 0.1, 0], 0.8) + _maxwellian(pl, 0.4, [-0.6, -0.15, 0], 1.2)
    lam, n = _stress_rate(pl, f)
    assert abs(lam / V.stress_rate_maxwell(1.5, n) - 1) > 0.02
