"""Pins of the DG element-collision oracle (Sec. 3.4: eqs. eq_massMatrix, eq_stiffMatrix3, HH and
the SVD variant eq_coln_derivation_SVD_3/4) against closed forms and the direct triple sum."""
import numpy as np
import pytest

import oracle as O
from oracle import dg as D


def test_lobatto_nodes_and_lagrange_basis():
    np.testing.assert_allclose(D.lobatto_nodes(2), [-1.0, 1.0])
    np.testing.assert_allclose(D.lobatto_nodes(3), [-1.0, 0.0, 1.0], atol=1e-15)
    np.testing.assert_allclose(D.lobatto_nodes(4), [-1.0, -1 / np.sqrt(5), 1 / np.sqrt(5), 1.0], atol=1e-15)
    for K in (2, 3, 5):
        nodes = D.lobatto_nodes(K)
        np.testing.assert_allclose(D.lagrange(nodes, nodes), np.eye(K), atol=1e-14)   # cardinal
        x = np.linspace(-1, 1, 11)
        np.testing.assert_allclose(D.lagrange(nodes, x).sum(0), 1.0, atol=1e-14)      # partition of unity


def test_mass_matrix_and_H_closed_forms():
    _, M2, H2 = D.dg_tensors(2)   # linear elements on [-1, 1]
    np.testing.assert_allclose(M2, [[2 / 3, 1 / 3], [1 / 3, 2 / 3]], atol=1e-15)
    np.testing.assert_allclose(H2[0, 0, 0], 1 / 2, atol=1e-15)
    np.testing.assert_allclose(H2[0, 0, 1], 1 / 6, atol=1e-15)
    np.testing.assert_allclose(H2[1, 0, 1], 1 / 6, atol=1e-15)
    np.testing.assert_allclose(H2[1, 1, 1], 1 / 2, atol=1e-15)
    _, M3, _ = D.dg_tensors(3)    # quadratic elements: (h / 30) [[4, 2, -1], [2, 16, 2], [-1, 2, 4]], h = 2
    np.testing.assert_allclose(M3, np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) / 15, atol=1e-15)


@pytest.mark.parametrize("K", [2, 3, 4, 5])
def test_H_symmetric_and_sums_to_mass_matrix(K):
    _, M, H = D.dg_tensors(K)
    for perm in ((0, 2, 1), (1, 0, 2), (2, 1, 0), (1, 2, 0), (2, 0, 1)):
        np.testing.assert_allclose(H, np.transpose(H, perm), atol=1e-15)
    np.testing.assert_allclose(H.sum(0), M, atol=1e-14)      # sum_m phi_m = 1
    np.testing.assert_allclose(M.sum(), 2.0, atol=1e-14)      # |element| = 2


def _element_inputs(K, N, L, seed):
    """K nodal distribution functions of one element: two-Maxwellian mixtures that vary across it."""
    rng = np.random.default_rng(seed)
    c = -L + (np.arange(N) + 0.5) * 2 * L / N
    cx, cy, cz = np.meshgrid(c, c, c, indexing="ij")
    F = np.empty((K, N, N, N))
    for l in range(K):
        f = 0
        for _ in range(2):
            n, T = rng.uniform(0.5, 1.5), rng.uniform(0.7, 1.3)
            u = rng.normal(0, 0.3, 3)
            f = f + n * (np.pi * T) ** -1.5 * np.exp(-((cx - u[0]) ** 2 + (cy - u[1]) ** 2 + (cz - u[2]) ** 2) / T)
        F[l] = f
    return F


@pytest.mark.parametrize("K", [2, 3])
def test_svd_variant_equals_direct_sum(K):
    """Eq. eq_coln_derivation_SVD_4 reproduces eq. HH to round-off when no singular value is cut."""
    plan = O.OraclePlan(8, 4.0, gamma=0.38, M=12, Nrho=8, nyquist="sym")
    _, _, H = D.dg_tensors(K)
    F = _element_inputs(K, 8, 4.0, 11 + K)
    direct = D.element_collision_direct(plan, H, F)
    svd = D.element_collision_svd(plan, H, F, 0.0)
    assert np.linalg.norm(svd - direct) <= 1e-12 * np.linalg.norm(direct)
    Us, Vs = D.svd_factors(H)
    for m in range(K):
        np.testing.assert_allclose(Us[m] @ Vs[m], H[m], atol=1e-14)
        assert Us[m].shape[1] <= K


def test_svd_truncation_drops_small_singular_values_only():
    _, _, H = D.dg_tensors(3)
    full = sum(u.shape[1] for u in D.svd_factors(H, 0.0)[0])
    cut = sum(u.shape[1] for u in D.svd_factors(H, 0.3)[0])
    assert cut < full
    for m, (u, v) in enumerate(zip(*D.svd_factors(H, 0.3))):
        s = np.linalg.svd(H[m], compute_uv=False)
        err = np.linalg.norm(u @ v - H[m], 2)
        dropped = s[s <= 0.3 * s[0]]
        assert err <= (dropped.max() if len(dropped) else 0.0) + 1e-14


@pytest.mark.parametrize("K,tol", [(2, 0.0), (3, 0.0), (3, 0.3)])
def test_symmetric_slices_eigen_form_equals_svd_variant(K, tol):
    """Every H[m] is symmetric, so its eigen-decomposition is an SVD: the signed sum of quadratic
    terms Q(f_r, f_r) equals eq. eq_coln_derivation_SVD_4 (and eq. HH without truncation)."""
    plan = O.OraclePlan(8, 4.0, gamma=0.38, M=12, Nrho=8, nyquist="sym")
    _, _, H = D.dg_tensors(K)
    F = _element_inputs(K, 8, 4.0, 31 + K)
    sym = D.element_collision_sym(plan, H, F, tol)
    svd = D.element_collision_svd(plan, H, F, tol)
    assert np.linalg.norm(sym - svd) <= 1e-12 * np.linalg.norm(svd)
    if tol == 0.0:
        direct = D.element_collision_direct(plan, H, F)
        assert np.linalg.norm(sym - direct) <= 1e-12 * np.linalg.norm(direct)
