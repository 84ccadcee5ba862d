"""FP64 CPU oracle of the fast Fourier spectral Boltzmann collision operator.

TEST INFRASTRUCTURE. Only tests/, the smoke check and bench.py's CPU-baseline leg may
import, call or execute this module. The GPU product path shares no code with it.

What it computes (arXiv:1809.10186, Appendix; "the paper" below):

  Q(f,g)(c) = int_{B_R} int_{S^2} B_sym(c_r, sigma.c_r_hat) [f(c') g(c'_*) - f(c) g(c - c_r)]
              d sigma d c_r,   c' = c - c_r/2 + c_r sigma/2,  c'_* = c - c_r/2 - c_r sigma/2
  (eq. apndx_Q), for the VHS kernel B = b |c_r|^gamma (eq. B_gen with alpha = 1), on the
  uniform cell-centred grid c_j = -L + (j + 1/2) dc, dc = 2L/N (Sec. 3.3), with f and g
  periodised on [-L, L]^3 and expanded in the truncated Fourier series with modes
  k in [-N/2, N/2 - 1]^3 (eq. summation).

Three evaluations are provided, each written from the definition it follows:

  direct_Q   (O1) the Galerkin sum  Q^_k = sum_{l+m=k} [G(l,m) - G(m,m)] f^_l g^_m
             with G from the quadrature form eq. lowrank1, O(N^6); tiny N only.
  fast_Q     (O3) the low-rank form eq. apndx_fs_Glm_Qk: for every radial node c_r and
             sphere point sigma the sum over l+m=k of (beta_r f^)_l (gamma_r g^)_m is a
             convolution, i.e. the DFT of a product of two translated grid functions;
             O(M N_rho) inverse DFTs, each a naive dense separable DFT (no FFT).
  G_exact    (O2) the kernel mode eq. GG with both sphere integrals done in closed form,
             leaving a 1-D radial integral evaluated with many Gauss-Legendre points.

Readings of the paper taken here (each one is listed in the design notes):

  * M counts the points of an antipodal FULL-sphere rule; the paper's half-sphere
    rule with M points is our rule with 2M points (its M = 6 is our M = 12).
  * Circular convolution: l + m is taken modulo N, the kernel factor is evaluated at
    the wrapped index, and, because the grid is cell-centred,
    e^{i pi (k +- N) c_j / L} = -e^{i pi k c_j / L}: a product mode that wraps picks up a
    factor -1 per wrapped axis. (This is what a grid-based FFT evaluation computes.)
  * Loss weight G(m,m) (loss="paper", default): eq. lowrank1 evaluated at l = m, where
    the sphere sum is exact, G(m,m) = 4 pi sum_r w_r F(2m, c_r). With it the oracle
    reproduces every entry of the paper's BKW error table (Sec. 4.3.1) to within ~30%.
    loss="conservative" uses G(-m, m) of eq. lowrank1 instead (equal for the exact
    kernel), built from the gain's own sphere rule, so that Q^_0 = 0 to round-off; its
    BKW errors are orders of magnitude above the paper's table, so it is not the default.
  * Nyquist modes: nyquist="paper" keeps the lattice exactly as written (the k = -N/2
    mode has no +N/2 partner, translates are complex, the result is Re Q);
    nyquist="sym" splits each Nyquist mode evenly between -N/2 and +N/2 so that every
    translate of a real grid function is real (its multiplier at k = -N/2 becomes
    cos(pi N t / 2L)). Both agree to round-off whenever f and g carry no Nyquist content.
  * SVD compression of the gain kernel: the N_rho columns of S(|k|, r) =
    sinc(pi c_r |k| / 2L), rows weighted by the square root of the multiplicity of |k|^2,
    truncated at a relative singular-value tolerance (svd_tol = 0: no truncation). The
    loss weight keeps the exact sinc (its argument 2|m| leaves the lattice's |k| range);
    in loss="conservative" mode the truncated S at |k| = 0 is used so mass stays exact.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np

from .quadrature import antipodal_pairs, gauss_legendre, sphere_rule

PI = math.pi


def b_vhs(omega: float) -> float:
    """Nondimensional VHS constant 1 / (2^{3-omega} Gamma(5/2 - omega) pi) (Sec. 2.1, alpha = 1)."""
    return 1.0 / (2.0 ** (3.0 - omega) * math.gamma(2.5 - omega) * PI)


def default_R(L: float) -> float:
    """Ball radius R = 4 L / (3 + sqrt 2) (Appendix, truncation of c_r)."""
    return 4.0 * L / (3.0 + math.sqrt(2.0))


@lru_cache(maxsize=8)
def _cached_sphere_rule(M):
    return sphere_rule(M)


class OraclePlan:
    """All parameters and FP64 tables of one discretisation (one N, L, kernel, rule)."""

    def __init__(self, N, L, gamma=0.0, b=None, R=None, M=12, Nrho=None, sphere=None,
                 svd_tol=0.0, svd_rank=0, nyquist="paper", loss="paper",
                 radial_factor=None):
        if N < 2 or N % 2:
            raise ValueError("N must be even")
        if nyquist not in ("paper", "sym"):
            raise ValueError("nyquist must be 'paper' or 'sym'")
        if loss not in ("paper", "conservative"):
            raise ValueError("loss must be 'paper' or 'conservative'")
        self.loss = loss
        self.N, self.L = int(N), float(L)
        self.gamma = float(gamma)
        self.b = b_vhs(1.0 - 0.5 * gamma) if b is None else float(b)
        self.R = default_R(L) if R is None else float(R)
        self.Nrho = int(Nrho) if Nrho else int(N)
        self.nyquist = nyquist
        self.dc = 2.0 * L / N
        # velocity grid (Sec. 3.3) and Fourier lattice (eq. summation)
        self.c = -L + (np.arange(N) + 0.5) * self.dc
        self.k = np.arange(-N // 2, N // 2)
        # per-axis DFT matrices of the paper's basis e^{i pi k c / L}
        self.E = np.exp(-1j * PI * np.outer(self.k, self.c) / L) / N    # f^_k = sum_j E[k,j] f_j
        self.Einv = np.exp(1j * PI * np.outer(self.c, self.k) / L)      # f_j = sum_k Einv[j,k] f^_k
        # radial Gauss-Legendre rule on [0, R]
        self.cr, self.wr = gauss_legendre(self.Nrho, 0.0, self.R)
        # sphere rule: one representative per antipodal pair, w = weight of each point
        if sphere is None:
            pts, wts, _ = _cached_sphere_rule(int(M))
        else:
            pts, wts = np.asarray(sphere[0], float), np.asarray(sphere[1], float)
        self.sigma, self.wsig = antipodal_pairs(pts, wts)
        self.M = 2 * len(self.sigma)
        # radial kernel factor rho_r = 4 pi b c_r^{gamma+2} (closed form of F for VHS, see F_closed)
        self.rho = 4.0 * PI * self.b * self.cr ** (self.gamma + 2.0)
        if radial_factor is not None:                       # e.g. ln c_r for d/d gamma
            self.rho = self.rho * np.asarray(radial_factor, float)
        kx, ky, kz = np.meshgrid(self.k, self.k, self.k, indexing="ij")
        self.k2 = (kx * kx + ky * ky + kz * kz).astype(np.int64)
        self.kabs = np.sqrt(self.k2.astype(np.float64))
        self.svd_tol, self.svd_rank = float(svd_tol), int(svd_rank)
        self._build_radial_kernel()
        self._build_loss_weight()

    # ---- kernel tables -------------------------------------------------------------

    def _build_radial_kernel(self):
        """S(|k|, r) = sinc(pi c_r |k| / 2L), optionally SVD-truncated; W_r(k) = w_r rho_r S."""
        q, inv, mult = np.unique(self.k2.ravel(), return_inverse=True, return_counts=True)
        kq = np.sqrt(q.astype(np.float64))
        S = np.sinc(np.outer(kq, self.cr) / (2.0 * self.L))     # np.sinc(x) = sin(pi x)/(pi x)
        self.svd_rank_used = self.Nrho
        if self.svd_tol > 0.0 or self.svd_rank > 0:
            sw = np.sqrt(mult.astype(np.float64))[:, None]
            U, sv, Vt = np.linalg.svd(sw * S, full_matrices=False)
            rank = self.svd_rank if self.svd_rank > 0 else int(np.sum(sv > self.svd_tol * sv[0]))
            rank = max(1, min(rank, len(sv)))
            S = (U[:, :rank] * sv[:rank]) @ Vt[:rank] / sw
            self.svd_rank_used = rank
        self.S_q = S                        # [distinct |k|^2, Nrho]
        self.S0 = S[0]                      # |k| = 0 row (q[0] == 0)
        S_lat = S[inv].reshape(self.N, self.N, self.N, self.Nrho)
        self.W = np.moveaxis(S_lat, -1, 0) * (self.wr * self.rho)[:, None, None, None]

    def mu(self, t: float) -> np.ndarray:
        """Per-axis translate multiplier for a shift t: e^{i pi k t / L} (Nyquist: see module doc)."""
        m = np.exp(1j * PI * self.k * t / self.L)
        if self.nyquist == "sym":
            m[0] = math.cos(PI * self.N * t / (2.0 * self.L))
        return m

    def mu3(self, s) -> np.ndarray:
        mx, my, mz = self.mu(s[0]), self.mu(s[1]), self.mu(s[2])
        return mx[:, None, None] * my[None, :, None] * mz[None, None, :]

    def shift(self, r: int, p: int) -> np.ndarray:
        """s_rp = c_r sigma_p / 2: the shift of the post-collision velocities (eq. apndx_Q)."""
        return 0.5 * self.cr[r] * self.sigma[p]

    def _build_loss_weight(self):
        """Loss multiplier G(m, m) on the lattice.

        loss="paper": eq. lowrank1 evaluated at l = m. Then l - m = 0, the sphere sum is
          sum_half w_sigma = 2 pi exactly and G(m,m) = 4 pi sum_r w_r F(2m, c_r)
          = 4 pi sum_r w_r rho_r sinc(pi c_r |m| / L): only the radial rule enters.
        loss="conservative": G(-m, m) of eq. lowrank1 (equal to G(m,m) for the exact kernel)
          built from the same translates as the gain,
          sum_r w_r rho_r S(0,r) sum_pairs w_p [mu_s(m)^2 + mu_{-s}(m)^2], which makes
          Q^_0 = 0 (mass conservation) hold to round-off for any sphere rule.
        """
        if self.loss == "paper":
            G = np.zeros((self.N,) * 3)
            for r in range(self.Nrho):
                G += 4.0 * PI * self.wr[r] * self.rho[r] * np.sinc(self.cr[r] * self.kabs / self.L)
            self.Gloss = G
            return
        G = np.zeros((self.N,) * 3, dtype=np.complex128)
        for r in range(self.Nrho):
            acc = np.zeros((self.N,) * 3, dtype=np.complex128)
            for p in range(len(self.sigma)):
                s = self.shift(r, p)
                acc += self.wsig[p] * (self.mu3(s) ** 2 + self.mu3(-s) ** 2)
            G += self.wr[r] * self.rho[r] * self.S0[r] * acc
        self.Gloss = G.real if self.nyquist == "sym" else G

    # ---- transforms (naive separable DFT, no FFT) -----------------------------------

    @staticmethod
    def _axis(mat, x, axis):
        return np.moveaxis(np.tensordot(mat, x, axes=([1], [axis])), 0, axis)

    def dft3(self, f):
        """f^_k = N^{-3} sum_j f_j e^{-i pi k.c_j / L}."""
        x = f.astype(np.complex128)
        for a in range(3):
            x = self._axis(self.E, x, a)
        return x

    def idft3(self, fh):
        """f(c_j) = sum_k f^_k e^{i pi k.c_j / L}."""
        x = fh
        for a in range(3):
            x = self._axis(self.Einv, x, a)
        return x

    def translate_hat(self, fh, s):
        """(T_s f)(c_j) = f^N(c_j + s): multiply every mode by its phase, transform back."""
        x = self.idft3(fh * self.mu3(s))
        return x.real if self.nyquist == "sym" else x


# ---- collision operator ---------------------------------------------------------------

def gain_radial_products(plan: OraclePlan, f, g):
    """P_r = sum_pairs w_p [(T_s f)(T_{-s} g) + (T_{-s} f)(T_s g)], s = c_r sigma_p / 2, per r."""
    fh = plan.dft3(f)
    gh = fh if g is f else plan.dft3(g)
    out = []
    for r in range(plan.Nrho):
        P = 0.0
        for p in range(len(plan.sigma)):
            s = plan.shift(r, p)
            fp, fm = plan.translate_hat(fh, s), plan.translate_hat(fh, -s)
            if g is f:
                gp, gm = fp, fm
            else:
                gp, gm = plan.translate_hat(gh, s), plan.translate_hat(gh, -s)
            P = P + plan.wsig[p] * (fp * gm + fm * gp)
        out.append(P)
    return out


def gain_Q(plan: OraclePlan, f, g):
    """Gain term: sum_r alpha_r(k) DFT(P_r)_k transformed back (eq. apndx_fs_Glm_Qk)."""
    Ph = 0.0
    for r, P in enumerate(gain_radial_products(plan, f, g)):
        Ph = Ph + plan.W[r] * plan.dft3(P)
    return plan.idft3(Ph)


def loss_Q(plan: OraclePlan, f, g):
    """Loss term f(c) (G(m,m) g^_m transformed back): a single convolution (Appendix)."""
    return f * plan.idft3(plan.Gloss * plan.dft3(g))


def fast_Q(plan: OraclePlan, f, g=None):
    """O3: bilinear Q(f, g) (Q(f, f) when g is None) on one grid, FP64; returns a real array."""
    f = np.asarray(f, dtype=np.float64)
    g = f if g is None else np.asarray(g, dtype=np.float64)
    return np.real(gain_Q(plan, f, g) - loss_Q(plan, f, g))


def fast_Q_batch(plan, F, G=None):
    F = np.asarray(F, dtype=np.float64)
    out = np.empty_like(F)
    for i in range(F.shape[0]):
        out[i] = fast_Q(plan, F[i], None if G is None else G[i])
    return out


def direct_Q(plan: OraclePlan, f, g=None, block=4096):
    """O1: the Galerkin sum with the quadrature kernel of eq. lowrank1, O(N^6) (paper lattice).

    Q^_k = sum_{l, m: l+m = k mod N} (-1)^{#wrapped axes} [Gq(l,m) - G_loss(m)] f^_l g^_m with
    Gq(l,m) = 2 sum_r w_r F(wrap(l+m), c_r) sum_pairs w_p cos(pi c_r (l-m).sigma_p / 2L),
    F(k, c_r) = rho_r S(|k|, r), and G_loss(m) = Gq(m,m) = 4 pi sum_r w_r F(2m, c_r)
    (loss="paper") or Gq(-m,m) (loss="conservative"); then Q_j = Re sum_k Q^_k e^{i pi k.c_j/L}.
    """
    if plan.nyquist != "paper":
        raise ValueError("direct_Q follows the paper's lattice (nyquist='paper')")
    N = plan.N
    f = np.asarray(f, dtype=np.float64)
    g = f if g is None else np.asarray(g, dtype=np.float64)
    fh = plan.dft3(f).ravel()
    gh = plan.dft3(g).ravel()
    kv = np.stack(np.meshgrid(plan.k, plan.k, plan.k, indexing="ij"), -1).reshape(-1, 3)
    nk = kv.shape[0]
    Wflat = plan.W.reshape(plan.Nrho, -1)                      # w_r rho_r S(|k|, r) on the lattice
    W0 = plan.wr * plan.rho * plan.S0                          # at k = 0
    cr, sig, ws = plan.cr, plan.sigma, plan.wsig
    Qh = np.zeros(nk, dtype=np.complex128)
    lidx = np.arange(nk)
    for m0 in range(0, nk, max(1, block // nk)):
        midx = np.arange(m0, min(nk, m0 + max(1, block // nk)))
        L_, M_ = np.meshgrid(lidx, midx, indexing="ij")
        l, m = kv[L_.ravel()], kv[M_.ravel()]
        ksum = l + m
        wraps = np.sum((ksum < -N // 2) | (ksum >= N // 2), axis=1)
        kw = (ksum + N // 2) % N - N // 2
        kidx = ((kw[:, 0] + N // 2) * N + (kw[:, 1] + N // 2)) * N + (kw[:, 2] + N // 2)
        diff = (l - m).astype(np.float64)
        # angular sums: sum_pairs w_p cos(pi c_r (l-m).sigma_p / 2L) and ... cos(pi c_r m.sigma_p / L)
        proj_d = diff @ sig.T                                  # [pairs_lm, npairs]
        proj_m = m.astype(np.float64) @ sig.T
        m_abs = np.linalg.norm(m.astype(np.float64), axis=1)
        gain_k = np.zeros(len(l))
        loss_k = np.zeros(len(l))
        for r in range(plan.Nrho):
            ang_g = np.cos(PI * cr[r] * proj_d / (2.0 * plan.L)) @ ws
            gain_k += 2.0 * Wflat[r, kidx] * ang_g
            if plan.loss == "paper":        # Gq(m, m): l - m = 0, half-sphere weights sum to 2 pi
                loss_k += 4.0 * PI * plan.wr[r] * F_closed(plan, 2.0 * m_abs, cr[r])
            else:                           # Gq(-m, m)
                ang_l = np.cos(PI * cr[r] * proj_m / plan.L) @ ws
                loss_k += 2.0 * W0[r] * ang_l
        sign = np.where(wraps % 2 == 1, -1.0, 1.0)
        contrib = sign * (gain_k - loss_k) * fh[L_.ravel()] * gh[M_.ravel()]
        np.add.at(Qh, kidx, contrib)
    return np.real(plan.idft3(Qh.reshape(N, N, N)))


def F_closed(plan: OraclePlan, k_abs, c_r):
    """F(k, c_r) of eq. realGG for VHS: 2 c_r^2 b c_r^gamma int_{S2+} cos(pi c_r k.c^/2L) dc^
    = 4 pi b c_r^{gamma+2} sinc(pi c_r |k| / 2L)."""
    return 4.0 * PI * plan.b * c_r ** (plan.gamma + 2.0) * np.sinc(c_r * k_abs / (2.0 * plan.L))


def G_exact(plan: OraclePlan, l, m, n_quad=400):
    """O2: kernel mode G(l, m) of eq. GG with exact sphere integrals:
    (4 pi)^2 b int_0^R c^{gamma+2} sinc(pi c |l+m| / 2L) sinc(pi c |l-m| / 2L) dc."""
    l = np.asarray(l, float)
    m = np.asarray(m, float)
    x, w = gauss_legendre(n_quad, 0.0, plan.R)
    a = np.linalg.norm(l + m)
    d = np.linalg.norm(l - m)
    integrand = x ** (plan.gamma + 2.0) * np.sinc(x * a / (2 * plan.L)) * np.sinc(x * d / (2 * plan.L))
    return (4.0 * PI) ** 2 * plan.b * np.sum(w * integrand)


def G_quadrature(plan: OraclePlan, l, m):
    """Gq(l, m) of eq. lowrank1 (no wrapping): 2 sum_r w_r F(l+m, c_r) sum_pairs w_p cos(...)."""
    l = np.asarray(l, float)
    m = np.asarray(m, float)
    a = np.linalg.norm(l + m)
    total = 0.0
    for r in range(plan.Nrho):
        ang = np.sum(plan.wsig * np.cos(PI * plan.cr[r] * (plan.sigma @ (l - m)) / (2.0 * plan.L)))
        total += 2.0 * plan.wr[r] * F_closed(plan, a, plan.cr[r]) * ang
    return total


# ---- derivatives ------------------------------------------------------------------------

def jvp(plan: OraclePlan, f, v):
    """Directional derivative of Q(f,f) along v: Q(f,v) + Q(v,f) (Q is bilinear)."""
    return fast_Q(plan, f, v) + fast_Q(plan, v, f)


def _apply_multiplier(plan, W, u):
    return np.real(plan.idft3(W * plan.dft3(u)))


def vjp(plan: OraclePlan, f, u):
    """Transpose of the Jacobian of Q(f,f) applied to u (real symmetric-Nyquist operator only).

    Q = sum_r K_r P_r - f (K_L f) with K_r, K_L real symmetric multipliers and
    P_r = sum_pairs 2 w_p (T_s f)(T_{-s} f); using T_s^T = T_{-s}:
    J^T u = sum_r sum_pairs 2 w_p [T_{-s}(K_r u . T_{-s} f) + T_s(K_r u . T_s f)]
            - u (K_L f) - K_L (u f).
    """
    if plan.nyquist != "sym":
        raise ValueError("vjp is defined for the real operator (nyquist='sym')")
    f = np.asarray(f, float)
    u = np.asarray(u, float)
    fh = plan.dft3(f)
    out = np.zeros_like(f)
    for r in range(plan.Nrho):
        ur = _apply_multiplier(plan, plan.W[r], u)
        for p in range(len(plan.sigma)):
            s = plan.shift(r, p)
            fp, fm = plan.translate_hat(fh, s), plan.translate_hat(fh, -s)
            out += 2.0 * plan.wsig[p] * (plan.translate_hat(plan.dft3(ur * fm), -s)
                                          + plan.translate_hat(plan.dft3(ur * fp), s))
    out -= u * _apply_multiplier(plan, plan.Gloss, f) + _apply_multiplier(plan, plan.Gloss, u * f)
    return out


def dgamma_plan(plan: OraclePlan) -> OraclePlan:
    """Plan whose radial factor is d rho_r / d gamma = ln(c_r) rho_r (b held fixed)."""
    return OraclePlan(plan.N, plan.L, gamma=plan.gamma, b=plan.b, R=plan.R, Nrho=plan.Nrho,
                      sphere=(np.concatenate([plan.sigma, -plan.sigma]),
                              np.concatenate([plan.wsig, plan.wsig])),
                      svd_tol=plan.svd_tol, svd_rank=plan.svd_rank, nyquist=plan.nyquist,
                      radial_factor=np.log(plan.cr))


def dQ_dgamma(plan: OraclePlan, f):
    """Derivative of Q(f,f) with respect to the VHS exponent gamma at fixed b."""
    return fast_Q(dgamma_plan(plan), f)


# ---- BKW closed form (Sec. 4.3, eqs. bkw_f and bkw_Q) ------------------------------------

def bkw_K(t):
    return 1.0 - math.exp(-t / 6.0)


def bkw_f(c2, t):
    """BKW solution for B = 1/(4 pi): unit density, unit temperature (eq. bkw_f); c2 = |c|^2."""
    K = bkw_K(t)
    return (np.exp(-c2 / (2 * K)) / (2 * (2 * PI * K) ** 1.5)
            * ((5 * K - 3) / K + (1 - K) / K ** 2 * c2))


def bkw_Q(c2, t):
    """Exact Q(f, f) = df/dt of the BKW solution (eq. bkw_Q)."""
    K = bkw_K(t)
    dK = math.exp(-t / 6.0) / 6.0
    f = bkw_f(c2, t)
    g = np.exp(-c2 / (2 * K)) / (2 * (2 * PI * K) ** 1.5) * (3 / K ** 2 + (K - 2) / K ** 3 * c2)
    return dK * ((-1.5 / K + c2 / (2 * K * K)) * f + g)


def grid_c2(plan: OraclePlan):
    cx, cy, cz = np.meshgrid(plan.c, plan.c, plan.c, indexing="ij")
    return cx * cx + cy * cy + cz * cz


# ---- moments and time stepping -------------------------------------------------------------

def moments(plan: OraclePlan, f):
    """Mid-point-rule moments (Sec. 3.3): n, u, T (= 2/(3n) int f |c-u|^2), P, q."""
    f = np.asarray(f, float)
    dv = plan.dc ** 3
    cx, cy, cz = np.meshgrid(plan.c, plan.c, plan.c, indexing="ij")
    C = np.stack([cx, cy, cz])
    n = f.sum() * dv
    u = (C * f).reshape(3, -1).sum(1) * dv / n
    d = C - u[:, None, None, None]
    d2 = (d * d).sum(0)
    T = 2.0 / (3.0 * n) * (f * d2).sum() * dv
    P = 2.0 * np.einsum("aijk,bijk,ijk->ab", d, d, f) * dv
    q = (d * d2 * f).reshape(3, -1).sum(1) * dv
    return {"n": n, "u": u, "T": T, "P": P, "q": q}


def conserved_moments(plan: OraclePlan, q):
    """(mass, momentum[3], energy) of a collision-operator output, mid-point rule."""
    dv = plan.dc ** 3
    cx, cy, cz = np.meshgrid(plan.c, plan.c, plan.c, indexing="ij")
    return (q.sum() * dv, np.array([(q * cx).sum(), (q * cy).sum(), (q * cz).sum()]) * dv,
            (q * (cx * cx + cy * cy + cz * cz)).sum() * dv)


def ssp_rk2(plan: OraclePlan, f, dt, steps):
    """Space-homogeneous df/dt = Q(f,f) with the 2nd-order SSP Runge-Kutta scheme (eq. SSPRK2)."""
    f = np.asarray(f, float).copy()
    for _ in range(steps):
        v1 = f + dt * fast_Q(plan, f)
        f = 0.5 * f + 0.5 * v1 + 0.5 * dt * fast_Q(plan, v1)
    return f


def ssp_rk3(plan: OraclePlan, f, dt, steps):
    """Space-homogeneous df/dt = Q(f,f) with the 3rd-order SSP Runge-Kutta scheme (eq. SSPRK3)."""
    f = np.asarray(f, float).copy()
    for _ in range(steps):
        v1 = f + dt * fast_Q(plan, f)
        v2 = 0.75 * f + 0.25 * v1 + 0.25 * dt * fast_Q(plan, v1)
        f = f / 3.0 + 2.0 / 3.0 * v2 + 2.0 / 3.0 * dt * fast_Q(plan, v2)
    return f


def entropy(plan: OraclePlan, f):
    """Boltzmann's H = int f ln f dc over the points where f > 0 (mid-point rule); the collision
    operator does not increase it (H-theorem)."""
    f = np.asarray(f, float)
    pos = f > 0
    return float((f[pos] * np.log(f[pos])).sum() * plan.dc ** 3)
