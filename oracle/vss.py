"""FP64 oracle of the collision operator for the variable soft sphere (VSS) kernel.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import or run anything in this package. The CUDA product path never does.

Kernel (arXiv:1809.10186, Sec. 2.1 eq. B_gen, in the nondimensional form of Sec. 2.2):

    B(c_r, cos chi) = b c_r^gamma (1 + cos chi)^(alpha - 1),    gamma = 2 (1 - omega),
    b = alpha / (2^(2 - omega + alpha) Gamma(5/2 - omega) pi),

VHS for alpha = 1, VSS for alpha in (1, 2]. The method only sees the symmetrised kernel of the
Appendix, B_sym(c_r, t) = b c_r^gamma [(1 + t)^(alpha-1) + (1 - t)^(alpha-1)] / 2, t = cos chi.
Its angular part no longer drops out of eq. realGG, so the kernel factor keeps the sphere point:

    F(k, c_r, sigma) = 2 c_r^2 int_{S2+} B_sym(c_r, sigma.e) cos(pi c_r k.e / 2L) de,

and the quadrature of eq. lowrank1 gives one convolution per radial point AND sphere point in
eq. apndx_fs_Glm_Qk:

    gain^_k = sum_r sum_p w_r F(k, c_r, sigma_p) DFT[ w_p ((T_s f)(T_-s g) + (T_-s f)(T_s g)) ]_k,

s = c_r sigma_p / 2, (sigma_p, w_p) the half-sphere rule. With alpha = 1 the F factor does not
depend on sigma_p and this is the VHS gain of collision.gain_Q term by term.

Readings taken here (listed with the others in the design notes):
  * The loss weight keeps the paper reading of collision.py, eq. lowrank1 at l = m:
    G(m, m) = 2 sum_r w_r sum_p w_p F(2m, c_r, sigma_p)  (loss="paper"), or
    G(-m, m) = 2 sum_r w_r sum_p w_p F(0, c_r, sigma_p) cos(pi c_r m.sigma_p / L)  ("conservative").
  * F is evaluated at the signed (wrapped) lattice index, exactly as the VHS oracle does.
  * No compression of the kernel factor (the radial SVD of the VHS plan does not apply).

F by quadrature: the integrand is even in e, so the half-sphere integral is half the full-sphere
one. In coordinates about sigma, e = t sigma + sqrt(1 - t^2)(cos phi u + sin phi v) with u along
the part of k orthogonal to sigma, k.e = |k| (mu t + nu sqrt(1 - t^2) cos phi), mu = sigma.k/|k|,
nu = sqrt(1 - mu^2). The phi integral of cos(A + Z cos phi) is 2 pi cos(A) J0(Z) (Bessel's
integral); the t integral of each half of B_sym is a Gauss-Jacobi rule with the weight
(1 + t)^(alpha-1) or (1 - t)^(alpha-1), which leaves a smooth integrand.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import j0, roots_jacobi

from .collision import OraclePlan

PI = math.pi


def b_vss(omega: float, alpha: float) -> float:
    """Nondimensional kernel constant alpha / (2^(2 - omega + alpha) Gamma(5/2 - omega) pi) (Sec. 2.2)."""
    return alpha / (2.0 ** (2.0 - omega + alpha) * math.gamma(2.5 - omega) * PI)


def B_sym(b: float, gamma: float, alpha: float, c_r, t):
    """Symmetrised kernel of the Appendix: b c_r^gamma [(1+t)^(alpha-1) + (1-t)^(alpha-1)] / 2."""
    t = np.asarray(t, float)
    return b * np.asarray(c_r, float) ** gamma * 0.5 * ((1.0 + t) ** (alpha - 1.0) + (1.0 - t) ** (alpha - 1.0))


def F_vss(b, gamma, alpha, L, k_abs, mu, c_r, n_t=None):
    """F(k, c_r, sigma) of eq. realGG for the VSS kernel; k_abs = |k|, mu = sigma.k/|k| (arrays).

    F = c_r^2 int_{-1}^{1} B_sym(c_r, t) 2 pi cos(a mu t) J0(a nu sqrt(1 - t^2)) dt,
    a = pi c_r |k| / 2L, each half of B_sym integrated with its own Gauss-Jacobi rule."""
    k_abs = np.asarray(k_abs, float)
    mu = np.clip(np.asarray(mu, float), -1.0, 1.0)
    a = PI * c_r * k_abs / (2.0 * L)
    if n_t is None:
        n_t = int(np.max(a, initial=0.0)) + 40
    t, w = roots_jacobi(n_t, 0.0, alpha - 1.0)          # weight (1 + t)^(alpha - 1) on [-1, 1]
    nu = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    A, MU, NU = a[..., None], mu[..., None], nu[..., None]

    def h(tt):   # 2 pi cos(a mu t) J0(a nu sqrt(1 - t^2)): the phi integral of cos(pi c_r k.e / 2L)
        return 2.0 * PI * np.cos(A * MU * tt) * j0(A * NU * np.sqrt(np.maximum(0.0, 1.0 - tt * tt)))

    # (1 - t)^(alpha-1) half: substitute t -> -t, which maps it onto the same weight
    integral = 0.5 * (h(t) @ w + h(-t) @ w)
    return c_r * c_r * b * c_r ** gamma * integral


class VSSPlan(OraclePlan):
    """An OraclePlan whose gain kernel factor depends on the sphere point (alpha != 1 allowed).

    Tables: A[r][p] (lattice) = w_r F(k, c_r, sigma_p) and the loss weight Gloss."""

    def __init__(self, N, L, gamma=0.0, alpha=1.0, b=None, **kw):
        if kw.get("svd_tol", 0.0) or kw.get("svd_rank", 0):
            raise ValueError("the VSS gain factor is not compressed")
        if not 1.0 <= alpha <= 2.0:
            raise ValueError("alpha must lie in [1, 2] (Sec. 2.1)")
        self.alpha = float(alpha)
        omega = 1.0 - 0.5 * gamma
        super().__init__(N, L, gamma=gamma, b=b_vss(omega, alpha) if b is None else b, **kw)

    def F(self, k_abs, mu, c_r):
        return F_vss(self.b, self.gamma, self.alpha, self.L, k_abs, mu, c_r)

    def _lattice_mu(self, kvec, p):
        """sigma_p . k/|k| on a [..., 3] array of lattice vectors (0 at k = 0)."""
        kk = np.linalg.norm(kvec, axis=-1)
        return np.where(kk > 0, (kvec @ self.sigma[p]) / np.where(kk > 0, kk, 1.0), 0.0), kk

    def _build_radial_kernel(self):
        kv = np.stack(np.meshgrid(self.k, self.k, self.k, indexing="ij"), -1).astype(np.float64)
        self.svd_rank_used = self.Nrho
        self.A = np.empty((self.Nrho, len(self.sigma)) + (self.N,) * 3)
        for p in range(len(self.sigma)):
            mu, kk = self._lattice_mu(kv, p)
            for r in range(self.Nrho):
                self.A[r, p] = self.wr[r] * self.F(kk, mu, self.cr[r])
        self.S0 = np.ones(self.Nrho)

    def _build_loss_weight(self):
        kv = np.stack(np.meshgrid(self.k, self.k, self.k, indexing="ij"), -1).astype(np.float64)
        G = np.zeros((self.N,) * 3, dtype=np.complex128 if self.loss == "conservative" else np.float64)
        for r in range(self.Nrho):
            if self.loss == "paper":            # eq. lowrank1 at l = m: F at 2m, weights over the half sphere
                for p in range(len(self.sigma)):
                    mu, kk = self._lattice_mu(2.0 * kv, p)
                    G += 2.0 * self.wr[r] * self.wsig[p] * self.F(kk, mu, self.cr[r])
            else:                               # G(-m, m): F at 0 (isotropic), the translates' phases
                F0 = float(self.F(np.zeros(1), np.zeros(1), self.cr[r])[0])
                acc = np.zeros((self.N,) * 3, dtype=np.complex128)
                for p in range(len(self.sigma)):
                    s = self.shift(r, p)
                    acc += self.wsig[p] * (self.mu3(s) ** 2 + self.mu3(-s) ** 2)
                G += self.wr[r] * F0 * acc
        self.Gloss = G.real if (self.loss == "paper" or self.nyquist == "sym") else G


def gain_Q_vss(plan: VSSPlan, f, g):
    """Gain of eq. apndx_fs_Glm_Qk with the sphere-dependent factor: one DFT per (r, p)."""
    fh = plan.dft3(f)
    gh = fh if g is f else plan.dft3(g)
    Ph = 0.0
    for r in range(plan.Nrho):
        for p in range(len(plan.sigma)):
            s = plan.shift(r, p)
            fp, fm = plan.translate_hat(fh, s), plan.translate_hat(fh, -s)
            if g is f:
                gp, gm = fp, fm
            else:
                gp, gm = plan.translate_hat(gh, s), plan.translate_hat(gh, -s)
            Ph = Ph + plan.A[r, p] * plan.dft3(plan.wsig[p] * (fp * gm + fm * gp))
    return plan.idft3(Ph)


def fast_Q_vss(plan: VSSPlan, f, g=None):
    """Bilinear Q(f, g) (Q(f, f) when g is None) for the VSS kernel, FP64, real."""
    f = np.asarray(f, dtype=np.float64)
    g = f if g is None else np.asarray(g, dtype=np.float64)
    loss = f * plan.idft3(plan.Gloss * plan.dft3(g))
    return np.real(gain_Q_vss(plan, f, g) - loss)


def direct_Q_vss(plan: VSSPlan, f, g=None):
    """The Galerkin sum with the sphere-dependent quadrature kernel of eq. lowrank1, O(N^6):

    Q^_k = sum_{l + m = k mod N} (-1)^{#wrapped axes} [Gq(l, m) - G_loss(m)] f^_l g^_m,
    Gq(l, m) = 2 sum_r w_r sum_p w_p F(wrap(l + m), c_r, sigma_p) cos(pi c_r (l - m).sigma_p / 2L),
    G_loss(m) = Gq(m, m) (loss="paper") or Gq(-m, m) (loss="conservative"); every F value is
    evaluated here afresh (paper lattice only; tiny N)."""
    if plan.nyquist != "paper":
        raise ValueError("direct_Q_vss follows the paper's lattice (nyquist='paper')")
    N = plan.N
    f = np.asarray(f, dtype=np.float64)
    g = f if g is None else np.asarray(g, dtype=np.float64)
    fh = plan.dft3(f).ravel()
    gh = plan.dft3(g).ravel()
    kv = np.stack(np.meshgrid(plan.k, plan.k, plan.k, indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    nk = len(kv)

    def Fk(kvecs, r, p):   # F(k, c_r, sigma_p) for an array of lattice vectors
        kk = np.linalg.norm(kvecs, axis=-1)
        mu = np.where(kk > 0, (kvecs @ plan.sigma[p]) / np.where(kk > 0, kk, 1.0), 0.0)
        return plan.F(kk, mu, plan.cr[r])

    # G_loss(m) for every lattice m
    Gl = np.zeros(nk)
    for r in range(plan.Nrho):
        for p in range(len(plan.sigma)):
            if plan.loss == "paper":
                Gl += 2.0 * plan.wr[r] * plan.wsig[p] * Fk(2.0 * kv, r, p)
            else:
                Gl += (2.0 * plan.wr[r] * plan.wsig[p] * Fk(np.zeros((1, 3)), r, p)[0]
                       * np.cos(PI * plan.cr[r] * (kv @ plan.sigma[p]) / plan.L))
    Qh = np.zeros(nk, dtype=np.complex128)
    for li in range(nk):
        l = kv[li]
        ksum = l + kv                                   # every m at once
        wraps = np.sum((ksum < -N // 2) | (ksum >= N // 2), axis=1)
        kw = (ksum + N // 2) % N - N // 2
        kidx = ((kw[:, 0] + N // 2) * N + (kw[:, 1] + N // 2)) * N + (kw[:, 2] + N // 2)
        Gq = np.zeros(nk)
        for r in range(plan.Nrho):
            for p in range(len(plan.sigma)):
                ang = np.cos(PI * plan.cr[r] * ((l - kv) @ plan.sigma[p]) / (2.0 * plan.L))
                Gq += 2.0 * plan.wr[r] * plan.wsig[p] * Fk(kw, r, p) * ang
        sign = np.where(wraps % 2 == 1, -1.0, 1.0)
        np.add.at(Qh, kidx.astype(np.int64), sign * (Gq - Gl) * fh[li] * gh)
    return np.real(plan.idft3(Qh.reshape(N, N, N)))


def stress_rate_maxwell(alpha: float, n: float) -> float:
    """For Maxwell molecules (omega = 1) with the VSS angular factor, the deviatoric stress obeys
    dP/dt = -lam P with lam = (3/4) n int_{S2} B sin^2 chi d sigma = 3 alpha n / (Gamma(3/2)(alpha+1)(alpha+2));
    the heat flux decays at 2/3 of that rate. Derived from the collision invariants' weak form."""
    return 3.0 * alpha * n / (math.gamma(1.5) * (alpha + 1.0) * (alpha + 2.0))
