"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each pin is chosen so that a plausible mistake in the oracle fails at least one of them:
  * the paper's own BKW error table (Sec. 4.3.1) fixes the normalisation of the kernel
    (b, rho_r = 4 pi b c_r^{gamma+2}, the sinc arguments), the radius R, the loss weight
    and the sphere rule; a factor or a dropped term moves the errors by decades;
  * the direct O(N^6) Galerkin sum pins the fast form's convolution structure
    (translates, signs, wrapping, pair weights) by brute force;
  * closed-form and brute-force integrals pin F, G and the translate operator;
  * conservation, equilibrium, equivariance and bilinearity pin symmetries;
  * finite differences pin the derivatives.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle.quadrature import gauss_legendre, product_rule
from paper_1809_10186_gb300 import workloads as W


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _bkw_plan(N, Nr, **kw):
    return O.OraclePlan(N, 6.62, gamma=0.0, b=1.0 / (4.0 * math.pi), M=12, Nrho=Nr, **kw)


def _load_table(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "bkw_table1.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                v = line.split()
                rows.append((int(v[0]), int(v[1]), [float(x) for x in v[2:5]]))
    return rows


# ---- the paper's worked example ---------------------------------------------------------

@pytest.mark.parametrize("N", [8, 16, 24, 32])
def test_bkw_error_table_reproduced(N, golden_dir):
    """Every entry of the paper's BKW table for this N is matched within a factor 1.5.

    The paper's M = 6 half-sphere design is our 12-point icosahedral rule; the domain is
    [-6.62, 6.62]^3, R = 4L/(3+sqrt 2), B = 1/(4 pi).
    """
    for n, nr, errs in _load_table(golden_dir):
        if n != N:
            continue
        plan = _bkw_plan(N, nr, nyquist="sym")
        c2 = O.grid_c2(plan)
        for t0, ref in zip((5.5, 6.5, 10.0), errs):
            err = np.abs(O.fast_Q(plan, O.bkw_f(c2, t0)) - O.bkw_Q(c2, t0)).max()
            assert ref / 1.5 < err < ref * 1.5, (N, nr, t0, err, ref)


def test_bkw_closed_form_Q_is_time_derivative_of_f():
    c2 = np.linspace(0.0, 30.0, 301)
    for t in (5.5, 6.5, 10.0):
        h = 1e-4
        fd = (O.bkw_f(c2, t + h) - O.bkw_f(c2, t - h)) / (2 * h)
        np.testing.assert_allclose(O.bkw_Q(c2, t), fd, atol=1e-10)


def test_bkw_f_unit_density_and_temperature():
    plan = _bkw_plan(32, 8)
    f = O.bkw_f(O.grid_c2(plan), 5.5)
    m = O.moments(plan, f)
    assert m["n"] == pytest.approx(1.0, abs=1e-12)
    assert np.abs(m["u"]).max() < 1e-14
    # unit temperature in the (1/3) int c^2 f sense is T = 2 in the paper's convention
    assert m["T"] == pytest.approx(2.0, abs=1e-10)
    # the generator module builds the same datum
    np.testing.assert_allclose(W.bkw(32, 6.62, 5.5), f, rtol=1e-14, atol=1e-300)


def test_moments_of_a_drifting_maxwellian_closed_form():
    """Sec. 3.5's Maxwellian n (pi T)^{-3/2} exp(-|c - u|^2 / T) in the moments' convention
    (T = 2/(3n) int f |c-u|^2, P = 2 int f (c-u)(c-u), q = int f (c-u)|c-u|^2): P = n T I, q = 0,
    to the mid-point rule's spectral accuracy on a domain that holds the tails."""
    plan = O.OraclePlan(32, 8.0, M=6, Nrho=4)
    n, u, T = 1.3, np.array([0.4, -0.25, 0.15]), 0.9
    f = W.maxwellian(32, 8.0, n, u, T)
    m = O.moments(plan, f)
    assert m["n"] == pytest.approx(n, rel=1e-12)
    np.testing.assert_allclose(m["u"], u, atol=1e-12)
    assert m["T"] == pytest.approx(T, rel=1e-12)
    np.testing.assert_allclose(m["P"], n * T * np.eye(3), atol=1e-12)
    np.testing.assert_allclose(m["q"], 0.0, atol=1e-12)


def test_moments_of_a_two_maxwellian_mixture_closed_form():
    """A mixture sum_i n_i M(u_i, T_i) with d_i = u_i - u (u the mixture's mean velocity):
    P = sum_i n_i T_i I + 2 sum_i n_i d_i d_i^T (off-diagonal terms from the drifts) and
    q = sum_i n_i d_i (5 T_i / 2 + |d_i|^2), from the Gaussian moments int M w_a w_b = n T/2 delta_ab,
    int M |w|^2 = 3 n T / 2 and the vanishing odd moments."""
    N, L = 40, 9.0
    plan = O.OraclePlan(N, L, M=6, Nrho=4)
    comps = [(0.7, np.array([0.5, -0.3, 0.2]), 1.1), (1.2, np.array([-0.4, 0.35, -0.1]), 0.8)]
    f = sum(W.maxwellian(N, L, n, u, T) for n, u, T in comps)
    ntot = sum(n for n, _, _ in comps)
    umix = sum(n * u for n, u, _ in comps) / ntot
    P = np.zeros((3, 3))
    q = np.zeros(3)
    for n, u, T in comps:
        d = u - umix
        P += n * T * np.eye(3) + 2.0 * n * np.outer(d, d)
        q += n * d * (2.5 * T + d @ d)
    m = O.moments(plan, f)
    assert m["n"] == pytest.approx(ntot, rel=1e-12)
    np.testing.assert_allclose(m["u"], umix, atol=1e-12)
    assert m["T"] == pytest.approx(np.trace(P) / (3.0 * ntot), rel=1e-12)
    np.testing.assert_allclose(m["P"], P, atol=1e-11)
    assert abs(m["P"][0, 1]) > 0.05 and abs(m["P"][1, 2]) > 0.01     # the drifts make it anisotropic
    np.testing.assert_allclose(m["q"], q, atol=1e-11)
    assert np.abs(q).min() > 0.01


def test_bkw_ssp_rk2_time_stepping():
    """20 SSP-RK2 steps of dt = 0.01 from t0 = 5.5 follow the closed form to Q-error level."""
    plan = _bkw_plan(24, 24, nyquist="sym")
    c2 = O.grid_c2(plan)
    f = O.ssp_rk2(plan, O.bkw_f(c2, 5.5), 0.01, 20)
    err = np.abs(f - O.bkw_f(c2, 5.7)).max()
    assert err < 0.2 * 2.42e-5 * 1.5 + 1e-7


def test_bkw_ssp_rk3_time_stepping_and_temporal_orders():
    """Eq. SSPRK3 follows the BKW closed form like eq. SSPRK2, and the two schemes converge in dt
    at orders 3 and 2 (self-convergence against dt/8: the spatial error is the same in every run)."""
    plan = _bkw_plan(16, 16, nyquist="sym")
    c2 = O.grid_c2(plan)
    f0 = O.bkw_f(c2, 5.5)
    f3 = O.ssp_rk3(plan, f0, 0.01, 20)
    f2 = O.ssp_rk2(plan, f0, 0.01, 20)
    ref_err = np.abs(f2 - O.bkw_f(c2, 5.7)).max()
    assert np.abs(f3 - O.bkw_f(c2, 5.7)).max() < 1.05 * ref_err + 1e-9
    T, dts = 2.0, (0.5, 0.25)
    for scheme, order in ((O.ssp_rk2, 2), (O.ssp_rk3, 3)):
        fine = scheme(plan, f0, 0.0625, int(T / 0.0625))
        e = [np.abs(scheme(plan, f0, dt, int(T / dt)) - fine).max() for dt in dts]
        rate = np.log2(e[0] / e[1])
        assert abs(rate - order) < 0.35, (order, e, rate)


def test_entropy_of_a_maxwellian_and_H_theorem():
    """H of n (pi T)^{-3/2} e^{-|c-u|^2/T} is n [ln(n (pi T)^{-3/2}) - 3/2]; under the collision
    operator H does not increase along an SSP-RK2 run from a two-Maxwellian mixture."""
    plan = O.OraclePlan(16, 6.0, gamma=0.38, M=12, Nrho=16, nyquist="sym")
    cx, cy, cz = np.meshgrid(plan.c, plan.c, plan.c, indexing="ij")
    n, T, u = 1.3, 0.9, np.array([0.2, -0.1, 0.05])
    fm = n * (np.pi * T) ** -1.5 * np.exp(-((cx - u[0]) ** 2 + (cy - u[1]) ** 2 + (cz - u[2]) ** 2) / T)
    # mid-point rule on the 16-point grid: spectrally accurate, 2e-6 here
    assert O.entropy(plan, fm) == pytest.approx(n * (np.log(n * (np.pi * T) ** -1.5) - 1.5), rel=1e-5)
    f = fm + 0.7 * (np.pi * 0.6) ** -1.5 * np.exp(-((cx + 1.0) ** 2 + cy ** 2 + cz ** 2) / 0.6)
    hs = [O.entropy(plan, f)]
    for _ in range(4):
        f = O.ssp_rk2(plan, f, 0.05, 1)
        hs.append(O.entropy(plan, f))
    assert all(b < a for a, b in zip(hs, hs[1:])), hs


# ---- direct Galerkin sum versus the fast form -------------------------------------------

@pytest.mark.parametrize("N,M,loss", [(4, 6, "paper"), (6, 12, "paper"), (8, 12, "paper"),
                                      (6, 26, "conservative"), (8, 6, "conservative")])
def test_direct_sum_equals_fast_form(N, M, loss):
    g_ = W.rng(100 + N)
    f = g_.random((N, N, N))
    g = g_.random((N, N, N))
    plan = O.OraclePlan(N, 3.3, gamma=0.38, M=M, Nrho=5, nyquist="paper", loss=loss)
    d = O.direct_Q(plan, f, g)
    assert _rel(O.fast_Q(plan, f, g), d) < 1e-12
    assert _rel(O.fast_Q(plan, f), O.direct_Q(plan, f)) < 1e-12


def test_direct_sum_equals_fast_form_with_svd_truncation():
    N = 8
    f = W.rough(1, N, 3)[0]
    plan = O.OraclePlan(N, 3.0, gamma=0.52, M=12, Nrho=8, svd_rank=3, nyquist="paper")
    assert plan.svd_rank_used == 3
    assert _rel(O.fast_Q(plan, f), O.direct_Q(plan, f)) < 1e-12


# ---- kernel modes and translates ---------------------------------------------------------

def test_F_closed_form_against_half_sphere_quadrature():
    plan = O.OraclePlan(8, 4.0, gamma=0.38, M=6, Nrho=4)
    z, wz = gauss_legendre(60, 0.0, 1.0)            # half sphere z >= 0
    phi = (np.arange(120) + 0.5) * 2 * math.pi / 120
    Z, P = np.meshgrid(z, phi, indexing="ij")
    s = np.sqrt(1 - Z * Z)
    X, Y = s * np.cos(P), s * np.sin(P)
    Wt = wz[:, None] * (2 * math.pi / 120)
    for kvec in ([0, 0, 0], [1, 0, 0], [2, -1, 3], [-4, 3, 1]):
        for cr in (0.3, 1.7, 3.1):
            arg = math.pi * cr * (kvec[0] * X + kvec[1] * Y + kvec[2] * Z) / (2 * plan.L)
            bf = 2 * cr ** 2 * plan.b * cr ** plan.gamma * np.sum(Wt * np.cos(arg))
            assert O.F_closed(plan, np.linalg.norm(kvec), cr) == pytest.approx(bf, rel=1e-11, abs=1e-14)


def test_G_exact_against_brute_force_eq_GG():
    """Eq. GG integrated numerically over B_R x S^2 (product rules) equals the closed radial form."""
    plan = O.OraclePlan(8, 4.0, gamma=0.52, M=6, Nrho=4)
    x, wx = gauss_legendre(40, 0.0, plan.R)
    z, wz = gauss_legendre(24, -1.0, 1.0)
    phi = (np.arange(48) + 0.5) * 2 * math.pi / 48
    Z, P = np.meshgrid(z, phi, indexing="ij")
    s = np.sqrt(1 - Z * Z)
    dirs = np.stack([s * np.cos(P), s * np.sin(P), Z], -1).reshape(-1, 3)
    wd = (wz[:, None] * np.full(48, 2 * math.pi / 48)).ravel()
    for l, m in (([1, 0, 0], [0, 1, 0]), ([2, -1, 0], [1, 1, -1]), ([0, 0, 0], [1, 2, 0])):
        l, m = np.array(l, float), np.array(m, float)
        total = 0.0
        for cr, w in zip(x, wx):
            ph_r = np.exp(-1j * math.pi * cr * (dirs @ (l + m)) / (2 * plan.L))   # over c_r direction
            ph_s = np.exp(1j * math.pi * cr * (dirs @ (l - m)) / (2 * plan.L))    # over sigma
            total += w * cr ** 2 * plan.b * cr ** plan.gamma * np.sum(wd * ph_r) * np.sum(wd * ph_s)
        ge = O.G_exact(plan, l, m)
        assert abs(total.imag) < 1e-10 * abs(ge)
        assert total.real == pytest.approx(ge, rel=1e-9)


def test_quadrature_kernel_converges_to_exact_kernel():
    l, m = np.array([2.0, -1.0, 0.0]), np.array([1.0, 1.0, -1.0])
    errs = []
    for M, nr in ((6, 4), (12, 8), (26, 16), (38, 32), ("product", 48)):
        sph = product_rule(30, 60) if M == "product" else None
        plan = O.OraclePlan(8, 4.0, gamma=0.38, M=12 if sph else M, Nrho=nr, sphere=sph)
        errs.append(abs(O.G_quadrature(plan, l, m) - O.G_exact(plan, l, m)) / abs(O.G_exact(plan, l, m)))
    assert errs[-1] < 1e-10 and errs == sorted(errs, reverse=True)


@pytest.mark.parametrize("nyquist", ["paper", "sym"])
def test_translate_of_band_limited_mode_is_exact_shift(nyquist):
    N, L = 8, 3.0
    plan = O.OraclePlan(N, L, M=6, Nrho=2, nyquist=nyquist)
    cx, cy, cz = np.meshgrid(plan.c, plan.c, plan.c, indexing="ij")
    k = np.array([3, -2, 1])                      # no Nyquist component
    s = np.array([0.37, -1.21, 2.05])
    f = np.cos(math.pi * (k[0] * cx + k[1] * cy + k[2] * cz) / L + 0.3)
    want = np.cos(math.pi * (k[0] * (cx + s[0]) + k[1] * (cy + s[1]) + k[2] * (cz + s[2])) / L + 0.3)
    np.testing.assert_allclose(np.real(plan.translate_hat(plan.dft3(f), s)), want, atol=1e-13)


def test_symmetric_translate_is_shift_of_real_trigonometric_interpolant():
    """nyquist='sym': T_s f equals the real interpolant (cos/sin basis with the Nyquist
    sine mode) evaluated at c_j + s, built here by solving the interpolation system."""
    N, L = 8, 2.5
    plan = O.OraclePlan(N, L, M=6, Nrho=2, nyquist="sym")

    def basis(c):
        cols = [np.ones_like(c)]
        for q in range(1, N // 2):
            cols += [np.cos(math.pi * q * c / L), np.sin(math.pi * q * c / L)]
        cols.append(np.sin(math.pi * (N // 2) * c / L))
        return np.stack(cols, -1)

    f = W.rough(1, N, 11)[0]
    s = np.array([0.41, -0.77, 1.93])
    mats = [basis(plan.c + s[a]) @ np.linalg.inv(basis(plan.c)) for a in range(3)]
    want = np.einsum("ai,bj,ck,ijk->abc", mats[0], mats[1], mats[2], f)
    got = plan.translate_hat(plan.dft3(f), s)
    assert np.abs(got - want).max() < 1e-12


def test_sym_and_paper_conventions_agree_without_nyquist_content():
    N, L = 8, 3.0
    f, g = W.rough(2, N, 5)
    p_pap = O.OraclePlan(N, L, gamma=0.52, M=12, Nrho=6, nyquist="paper")
    p_sym = O.OraclePlan(N, L, gamma=0.52, M=12, Nrho=6, nyquist="sym")

    def strip(x):                                   # remove every mode with a k_a = -N/2
        h = p_pap.dft3(x)
        h[0, :, :] = 0
        h[:, 0, :] = 0
        h[:, :, 0] = 0
        return np.real(p_pap.idft3(h))

    f0, g0 = strip(f), strip(g)
    assert _rel(O.fast_Q(p_sym, f0, g0), O.fast_Q(p_pap, f0, g0)) < 1e-12
    # with Nyquist content the two discretisations genuinely differ
    assert _rel(O.fast_Q(p_sym, f, g), O.fast_Q(p_pap, f, g)) > 1e-6


# ---- invariants ----------------------------------------------------------------------------

def test_conservative_loss_conserves_mass_to_round_off():
    N = 12
    f = W.rough(1, N, 9)[0]
    plan = O.OraclePlan(N, 4.0, gamma=0.38, M=12, Nrho=N, nyquist="sym", loss="conservative")
    q = O.fast_Q(plan, f)
    loss_mass = np.sum(np.abs(np.real(O.loss_Q(plan, f, f))))
    assert abs(np.sum(q)) < 1e-13 * loss_mass


@pytest.mark.slow
def test_moments_and_equilibrium_spectrally_small():
    N, L = 24, 6.0
    plan = O.OraclePlan(N, L, gamma=0.38, M=12, Nrho=N, nyquist="sym")
    F, _ = W.two_maxwellian(1, N, L, 7)
    q = O.fast_Q(plan, F[0])
    scale = O.conserved_moments(plan, np.abs(np.real(O.loss_Q(plan, F[0], F[0]))))
    mass, mom, energy = O.conserved_moments(plan, q)
    assert abs(mass) < 1e-6 * scale[0]
    assert np.abs(mom).max() < 1e-4 * scale[0]
    assert abs(energy) < 1e-5 * scale[2]
    mx = W.maxwellian(N, L, 1.0, np.array([0.1, -0.2, 0.05]), 1.0)
    lm = np.real(O.loss_Q(plan, mx, mx))
    assert np.abs(O.fast_Q(plan, mx)).max() < 1e-4 * np.abs(lm).max()


def test_integer_shift_equivariance():
    N = 8
    f = W.rough(1, N, 21)[0]
    plan = O.OraclePlan(N, 3.0, gamma=0.52, M=12, Nrho=6, nyquist="sym")
    sh = (2, -3, 5)
    q = O.fast_Q(plan, f)
    np.testing.assert_allclose(O.fast_Q(plan, np.roll(f, sh, axis=(0, 1, 2))),
                               np.roll(q, sh, axis=(0, 1, 2)), atol=1e-13 * np.abs(q).max())


@pytest.mark.parametrize("M", [6, 26])
def test_octahedral_equivariance(M):
    N = 8
    f = W.rough(1, N, 23)[0]
    plan = O.OraclePlan(N, 3.0, gamma=0.38, M=M, Nrho=6, nyquist="sym")
    q = O.fast_Q(plan, f)
    tol = 1e-13 * np.abs(q).max()
    np.testing.assert_allclose(O.fast_Q(plan, f.transpose(2, 0, 1)), q.transpose(2, 0, 1), atol=tol)
    np.testing.assert_allclose(O.fast_Q(plan, f[::-1]), q[::-1], atol=tol)


def test_bilinearity():
    N = 8
    f, h, g = W.rough(3, N, 31)
    plan = O.OraclePlan(N, 3.0, gamma=0.38, M=12, Nrho=5, nyquist="sym")
    a, b = 0.7, -1.9
    lhs = O.fast_Q(plan, a * f + b * h, g)
    rhs = a * O.fast_Q(plan, f, g) + b * O.fast_Q(plan, h, g)
    assert _rel(lhs, rhs) < 1e-13


# ---- derivatives ---------------------------------------------------------------------------

def test_jvp_equals_central_difference():
    N = 8
    f, v = W.rough(2, N, 41)
    plan = O.OraclePlan(N, 3.0, gamma=0.52, M=12, Nrho=6, nyquist="sym")
    h = 1e-3
    fd = (O.fast_Q(plan, f + h * v) - O.fast_Q(plan, f - h * v)) / (2 * h)
    assert _rel(O.jvp(plan, f, v), fd) < 1e-10          # exact: Q is quadratic


def test_vjp_is_transpose_of_jvp():
    N = 8
    f, v, u = W.rough(3, N, 43)
    plan = O.OraclePlan(N, 3.0, gamma=0.52, M=12, Nrho=6, nyquist="sym")
    lhs = np.sum(u * O.jvp(plan, f, v))
    rhs = np.sum(O.vjp(plan, f, u) * v)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_dgamma_equals_central_difference():
    N = 8
    f = W.rough(1, N, 47)[0]
    kw = dict(M=12, Nrho=6, nyquist="sym", b=0.05)
    gam, h = 0.52, 1e-4
    fd = (O.fast_Q(O.OraclePlan(N, 3.0, gamma=gam + h, **kw), f)
          - O.fast_Q(O.OraclePlan(N, 3.0, gamma=gam - h, **kw), f)) / (2 * h)
    assert _rel(O.dQ_dgamma(O.OraclePlan(N, 3.0, gamma=gam, **kw), f), fd) < 1e-7


def test_svd_truncation_error_tracks_tolerance():
    N = 16
    F, _ = W.two_maxwellian(1, N, 5.0, 3)
    base = O.OraclePlan(N, 5.0, gamma=0.52, M=12, Nrho=N, nyquist="sym")
    q0 = O.fast_Q(base, F[0])
    ref = np.linalg.norm(np.real(O.loss_Q(base, F[0], F[0])))
    for tol in (1e-4, 1e-8):
        p = O.OraclePlan(N, 5.0, gamma=0.52, M=12, Nrho=N, nyquist="sym", svd_tol=tol)
        assert p.svd_rank_used < N
        assert np.linalg.norm(O.fast_Q(p, F[0]) - q0) / ref < 10 * tol


# ---- the pins catch planted mistakes --------------------------------------------------------

def _bkw_err(plan):
    c2 = O.grid_c2(plan)
    return np.abs(O.fast_Q(plan, O.bkw_f(c2, 6.5)) - O.bkw_Q(c2, 6.5)).max()


def test_planted_mistakes_are_caught(monkeypatch):
    good = _bkw_err(_bkw_plan(24, 12, nyquist="sym"))
    assert good < 1.5 * 4.22e-6

    # (1) radial factor c_r^gamma instead of c_r^(gamma+2)
    p = _bkw_plan(24, 12, nyquist="sym")
    p.rho = p.rho / p.cr ** 2
    p._build_radial_kernel()
    p._build_loss_weight()
    assert _bkw_err(p) > 100 * good

    # (2) loss term dropped
    monkeypatch.setattr(O.collision, "loss_Q", lambda plan, f, g: 0.0 * f)
    assert _bkw_err(_bkw_plan(24, 12, nyquist="sym")) > 100 * good
    monkeypatch.undo()

    # (3) post-collision shift c_r sigma instead of c_r sigma / 2
    monkeypatch.setattr(O.OraclePlan, "shift", lambda self, r, q: self.cr[r] * self.sigma[q])
    assert _bkw_err(_bkw_plan(24, 12, nyquist="sym")) > 100 * good
    monkeypatch.undo()

    # (4) wrap sign of the cell-centred grid omitted from the direct sum
    N = 6
    f = W.rough(1, N, 5)[0]
    plan = O.OraclePlan(N, 3.0, gamma=0.3, M=6, Nrho=4)
    good_d = _rel(O.fast_Q(plan, f), O.direct_Q(plan, f))
    monkeypatch.setattr(O.collision.np, "where",
                        lambda c, a, b: np.ones_like(np.asarray(c, dtype=float)))
    bad_d = _rel(O.fast_Q(plan, f), O.direct_Q(plan, f))
    monkeypatch.undo()
    assert good_d < 1e-12 and bad_d > 1e-6
