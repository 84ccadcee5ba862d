"""FP64 oracle of the 1-D DGFS right-hand side: DG transport with the upwind flux, the fully diffuse
wall condition, and the element collision term (arXiv:1809.10186, Sec. 3.1 eq. eq_weakForm,
eq. eq_numericalFlux_upwind, Sec. 3.5 and the boundary condition of Sec. 3.6).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import or run anything in this package. The CUDA product path never does.

Geometry: x in [edges[0], edges[I]], I elements D^i = [edges[i], edges[i+1]] of width h_i, walls
at both ends with outward normals -x (left) and +x (right), each wall moving with u_w (no normal
component) at temperature T_w. In every element the distribution function is the nodal expansion
f^i(x, c) = sum_l F^i_l(c) phi_l(x) on the K Gauss-Lobatto points (eq. eq_DG_local_approx). With
M, S and H on the reference element [-1, 1] (eqs. eq_massMatrix, eq_stiffMatrix1, eq_stiffMatrix3;
the physical M and H carry the Jacobian h/2, S does not), eq. eq_weakForm reads

    (h/2) M dF/dt = c_1 S F - Fl + (1/Kn) (h/2) sum_{l1,l2} H Q(F_l1, F_l2),
    S[m][l] = int phi_l dphi_m/dxi,  Fl_m = phi_m(x_R) F*_R - phi_m(x_L) F*_L,

with the upwind flux F* = c_1 f(interior trace) where c_1 n >= 0 and c_1 f(exterior trace) where
c_1 n < 0. At a wall the exterior trace of the incoming velocities ((c - u_w).n < 0) is n_w f_w,
f_w = exp(-|c - u_w|^2 / T_w), and n_w balances the mass flux of the outgoing interior trace:
    n_w = - sum_{(c-u_w).n >= 0} (c - u_w).n f  /  sum_{(c-u_w).n < 0} (c - u_w).n f_w
(mid-point rule on the velocity grid; the cell volume cancels). Kn = inf drops the collision term.
"""
from __future__ import annotations

import math

import numpy as np

from .dg import dg_tensors, element_collision_direct, element_collision_svd, lagrange
from .quadrature import gauss_legendre


def stiffness(K: int) -> np.ndarray:
    """S[m][l] = int_{-1}^{1} phi_l(xi) phi_m'(xi) dxi on the K Gauss-Lobatto nodal basis (exact
    Gauss-Legendre quadrature of the degree 2K - 3 integrand; phi_m' from the polynomial)."""
    nodes, _, _ = dg_tensors(K)
    x, w = gauss_legendre(K + 1)
    phi = lagrange(nodes, x)                                   # [K][q]
    dphi = np.empty_like(phi)
    for m in range(K):
        others = np.delete(nodes, m)
        coef = np.poly(others) / np.prod(nodes[m] - others)   # phi_m as a monomial polynomial
        dphi[m] = np.polyval(np.polyder(coef), x)
    return np.einsum("lq,mq,q->ml", phi, dphi, w)


def wall_maxwellian(plan, u_w, T_w) -> np.ndarray:
    cx, cy, cz = np.meshgrid(plan.c, plan.c, plan.c, indexing="ij")
    return np.exp(-((cx - u_w[0]) ** 2 + (cy - u_w[1]) ** 2 + (cz - u_w[2]) ** 2) / T_w)


class SlabOracle:
    """RHS of the 1-D DG system for a collision oracle plan (OraclePlan or VSSPlan)."""

    def __init__(self, plan, K, edges, Kn, wall_left, wall_right, svd_tol=None, collide=None):
        self.plan, self.K = plan, int(K)
        self.edges = np.asarray(edges, float)
        self.I = len(self.edges) - 1
        self.h = np.diff(self.edges)
        self.Kn = float(Kn)
        self.nodes, self.M, self.H = dg_tensors(self.K)
        self.S = stiffness(self.K)
        self.Minv = np.linalg.inv(self.M)
        self.svd_tol = svd_tol
        self.collide = collide or (lambda H, F: element_collision_svd(plan, H, F, svd_tol) if svd_tol is not None
                                   else element_collision_direct(plan, H, F))
        self.set_walls(wall_left, wall_right)
        cx, _, _ = np.meshgrid(plan.c, plan.c, plan.c, indexing="ij")
        self.c1 = cx

    def set_walls(self, wall_left, wall_right):
        self.walls = []
        for w in (wall_left, wall_right):
            u, T = np.asarray(w[:3], float), float(w[3])
            if u[0] != 0.0:
                raise ValueError("walls move parallel to themselves (u_w . n = 0)")
            self.walls.append((u, T, wall_maxwellian(self.plan, u, T)))

    def wall_density(self, side, f_int):
        """n_w of the left (side 0, n = -x) or right (side 1, n = +x) wall for the interior trace f_int."""
        u, T, fw = self.walls[side]
        cn = -self.c1 if side == 0 else self.c1                   # (c - u_w) . n with u_w . n = 0
        out = cn >= 0
        return -np.sum(cn[out] * f_int[out]) / np.sum(cn[~out] * fw[~out])

    def traces(self, F):
        """Exterior traces at the left and right face of every element."""
        I, K = self.I, self.K
        left = [None] * I
        right = [None] * I
        for i in range(I):
            left[i] = F[i - 1][K - 1] if i > 0 else self.wall_density(0, F[0][0]) * self.walls[0][2]
            right[i] = F[i + 1][0] if i < I - 1 else self.wall_density(1, F[I - 1][K - 1]) * self.walls[1][2]
        return left, right

    def transport(self, F):
        """c_1 S F - Fl for every element (the transport part of the weak form, before (h/2) M)."""
        F = np.asarray(F, float)
        K, c1 = self.K, self.c1
        left, right = self.traces(F)
        out = np.empty_like(F)
        for i in range(self.I):
            fR = c1 * np.where(c1 >= 0, F[i][K - 1], right[i])    # right face, n = +1
            fL = c1 * np.where(-c1 >= 0, F[i][0], left[i])        # left face, n = -1
            for m in range(K):
                v = c1 * sum(self.S[m][l] * F[i][l] for l in range(K))
                if m == K - 1:
                    v = v - fR
                if m == 0:
                    v = v + fL
                out[i][m] = v
        return out

    def rhs(self, F):
        """dF/dt of eq. eq_weakForm for every element and node: [I][K][N][N][N]."""
        F = np.asarray(F, float)
        T = self.transport(F)
        out = np.empty_like(F)
        for i in range(self.I):
            C = self.collide(self.H, F[i]) if math.isfinite(self.Kn) else np.zeros_like(F[i])
            for m in range(self.K):
                out[i][m] = sum(self.Minv[m][l] * (2.0 / self.h[i] * T[i][l] + C[l] / self.Kn) for l in range(self.K))
        return out

    def ssp_rk2(self, F, dt, steps):
        F = np.asarray(F, float).copy()
        for _ in range(steps):
            v1 = F + dt * self.rhs(F)
            F = 0.5 * F + 0.5 * v1 + 0.5 * dt * self.rhs(v1)
        return F

    def ssp_rk3(self, F, dt, steps):
        F = np.asarray(F, float).copy()
        for _ in range(steps):
            v1 = F + dt * self.rhs(F)
            v2 = 0.75 * F + 0.25 * v1 + 0.25 * dt * self.rhs(v1)
            F = F / 3.0 + 2.0 / 3.0 * v2 + 2.0 / 3.0 * dt * self.rhs(v2)
        return F

    def node_positions(self):
        """Physical x of every DG node: [I][K]."""
        return np.array([0.5 * (a + b) + 0.5 * (b - a) * self.nodes for a, b in zip(self.edges[:-1], self.edges[1:])])

    def mass(self, F):
        """int int f dx dc over the slab: int phi_l dx = (h/2) sum_m M[m][l] (the basis sums to 1),
        the mid-point rule in c."""
        F = np.asarray(F, float)
        wl = self.M.sum(axis=0)
        return float(sum(0.5 * self.h[i] * np.tensordot(wl, F[i], axes=1).sum() for i in range(self.I))
                     * self.plan.dc ** 3)
