"""FP64 oracle of the DG element collision term (arXiv:1809.10186, Sec. 3.4).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import or run anything in this package. The CUDA product path never does.

In the weak form (eq. eq_weakForm) the collision term of test function m in element i is

    C_m(c) = sum_{l1, l2} H[m, l1, l2] Q(F_l1, F_l2)(c)                      (eq. HH)

with H[m, l1, l2] = int_D phi_m phi_l1 phi_l2 dx (eq. eq_stiffMatrix3), F_l the nodal values of
the distribution function and Q the bilinear collision operator. The SVD variant
(eqs. eq_coln_derivation_SVD_3 and _4) factors each K x K slice H[m] = sum_r U[l1, r] V[r, l2]
(singular values absorbed in V) and evaluates

    C_m = sum_r Q(f_r, g_r),   f_r = sum_l U[l, r] F_l,   g_r = sum_l V[r, l] F_l,

with R_m <= K terms instead of K^2. Readings taken here: the basis is the 1-D nodal Lagrange
basis on the K Gauss-Lobatto points of the reference element [-1, 1] (the paper's "conventional
nodal DG basis"; its 1-D cases use polynomial order K - 1 = 2); the rank R_m counts singular
values above svd_tol times the largest one of H[m] (svd_tol = 0 keeps every nonzero one).
"""
from __future__ import annotations

import numpy as np

from .collision import fast_Q
from .quadrature import gauss_legendre


def lobatto_nodes(K: int) -> np.ndarray:
    """The K Gauss-Lobatto points of [-1, 1]: the end points and the roots of P'_{K-1}."""
    if K < 2:
        raise ValueError("K >= 2")
    inner = np.polynomial.legendre.Legendre.basis(K - 1).deriv().roots() if K > 2 else np.array([])
    return np.concatenate([[-1.0], np.sort(np.real(inner)), [1.0]])


def lagrange(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """phi_l(x) for every node l (rows) and point x (columns): prod_{j != l} (x - x_j)/(x_l - x_j)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.ones((len(nodes), len(x)))
    for l, xl in enumerate(nodes):
        for j, xj in enumerate(nodes):
            if j != l:
                out[l] *= (x - xj) / (xl - xj)
    return out


def dg_tensors(K: int):
    """Nodes, mass matrix M[m, l] and tensor H[m, l1, l2] on [-1, 1] (eqs. eq_massMatrix and
    eq_stiffMatrix3), by Gauss-Legendre quadrature exact for the degree 3 (K - 1) integrands."""
    nodes = lobatto_nodes(K)
    x, w = gauss_legendre((3 * K) // 2 + 1)
    phi = lagrange(nodes, x)                                    # [K][q]
    M = np.einsum("mq,lq,q->ml", phi, phi, w)
    H = np.einsum("mq,aq,bq,q->mab", phi, phi, phi, w)
    return nodes, M, H


def element_collision_direct(plan, H: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Eq. HH: C[m] = sum_{l1, l2} H[m, l1, l2] Q(F[l1], F[l2]); F is [K][N][N][N]."""
    K = H.shape[0]
    Q = [[fast_Q(plan, F[a], F[b]) for b in range(K)] for a in range(K)]
    C = np.zeros_like(np.asarray(F, dtype=np.float64))
    for m in range(K):
        for a in range(K):
            for b in range(K):
                C[m] += H[m, a, b] * Q[a][b]
    return C


def svd_factors(H: np.ndarray, svd_tol: float = 0.0):
    """Eq. eq_coln_derivation_SVD_3 for every m: lists of U[m] (K x R_m) and V[m] (R_m x K)
    with the singular values absorbed in V, truncated at svd_tol relative to the largest."""
    Us, Vs = [], []
    for m in range(H.shape[0]):
        u, s, vt = np.linalg.svd(H[m])
        keep = s > (svd_tol * s[0] if svd_tol > 0 else 1e-14 * s[0])
        Us.append(u[:, keep])
        Vs.append(s[keep, None] * vt[keep])
    return Us, Vs


def element_collision_svd(plan, H: np.ndarray, F: np.ndarray, svd_tol: float = 0.0) -> np.ndarray:
    """Eq. eq_coln_derivation_SVD_4: C[m] = sum_r Q(f_r, g_r)."""
    F = np.asarray(F, dtype=np.float64)
    Us, Vs = svd_factors(H, svd_tol)
    C = np.zeros_like(F)
    for m in range(H.shape[0]):
        for r in range(Us[m].shape[1]):
            fr = np.tensordot(Us[m][:, r], F, axes=1)
            gr = np.tensordot(Vs[m][r], F, axes=1)
            C[m] += fast_Q(plan, fr, gr)
    return C


def element_collision_sym(plan, H: np.ndarray, F: np.ndarray, svd_tol: float = 0.0) -> np.ndarray:
    """Eq. eq_coln_derivation_SVD_4 for symmetric slices H[m] (the nodal basis gives them): the
    eigen-decomposition H[m] = sum_r lambda_r u_r u_r^T is an SVD with singular values |lambda_r|
    and V[r] = sign(lambda_r) |lambda_r| u_r^T, and Q is bilinear, so
    C[m] = sum_r sign(lambda_r) Q(f_r, f_r),  f_r = sqrt|lambda_r| sum_l u_r[l] F_l,
    truncated like the SVD (|lambda_r| above svd_tol times the largest)."""
    F = np.asarray(F, dtype=np.float64)
    C = np.zeros_like(F)
    for m in range(H.shape[0]):
        lam, U = np.linalg.eigh(H[m])
        top = np.abs(lam).max()
        for r in range(len(lam)):
            if abs(lam[r]) <= (svd_tol * top if svd_tol > 0 else 1e-14 * top):
                continue
            fr = np.sqrt(abs(lam[r])) * np.tensordot(U[:, r], F, axes=1)
            C[m] += np.sign(lam[r]) * fast_Q(plan, fr)
    return C

