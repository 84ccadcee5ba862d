"""Pins of the oracle's quadrature rules against closed forms (no GPU)."""
import math

import numpy as np
import pytest

from oracle.quadrature import (antipodal_pairs, gauss_legendre, rule_moment_errors,
                               sphere_monomial_integral, sphere_rule)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16, 32, 48])
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    R = 5.987
    x, w = gauss_legendre(n, 0.0, R)
    assert np.all((x > 0) & (x < R)) and np.all(w > 0)
    for d in range(2 * n):
        exact = R ** (d + 1) / (d + 1)
        assert abs(np.sum(w * x ** d) - exact) <= 1e-13 * exact * max(1, d)
    # not exact at degree 2n: the rule's degree is tight (the defect shrinks fast with n)
    if n <= 5:
        exact = R ** (2 * n + 1) / (2 * n + 1)
        assert abs(np.sum(w * x ** (2 * n)) - exact) > 1e-6 * exact


def test_gauss_legendre_two_point_closed_form():
    x, w = gauss_legendre(2, -1.0, 1.0)
    np.testing.assert_allclose(np.sort(x), [-1 / math.sqrt(3), 1 / math.sqrt(3)], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [1.0, 1.0], atol=1e-15)


def test_sphere_monomial_integrals_closed_forms():
    assert sphere_monomial_integral(0, 0, 0) == pytest.approx(4 * math.pi, rel=1e-15)
    assert sphere_monomial_integral(2, 0, 0) == pytest.approx(4 * math.pi / 3, rel=1e-15)
    assert sphere_monomial_integral(2, 2, 0) == pytest.approx(4 * math.pi / 15, rel=1e-15)
    assert sphere_monomial_integral(2, 2, 2) == pytest.approx(4 * math.pi / 105, rel=1e-15)
    assert sphere_monomial_integral(1, 2, 0) == 0.0
    # brute force with a fine product rule: GL in z, uniform in phi
    z, wz = gauss_legendre(40, -1.0, 1.0)
    phi = (np.arange(80) + 0.5) * 2 * math.pi / 80
    Z, P = np.meshgrid(z, phi, indexing="ij")
    s = np.sqrt(1 - Z * Z)
    X, Y = s * np.cos(P), s * np.sin(P)
    W = wz[:, None] * (2 * math.pi / 80)
    for a, b, c in [(4, 0, 0), (2, 4, 0), (0, 2, 6), (2, 2, 2), (4, 4, 2)]:
        bf = np.sum(W * X ** a * Y ** b * Z ** c)
        assert bf == pytest.approx(sphere_monomial_integral(a, b, c), rel=1e-13)


@pytest.mark.parametrize("M,degree", [(6, 3), (12, 5), (26, 7), (38, 9)])
def test_sphere_rules_exact_to_stated_degree(M, degree):
    pts, w, d = sphere_rule(M)
    assert d == degree and len(pts) == M
    np.testing.assert_allclose(np.linalg.norm(pts, axis=1), 1.0, atol=1e-15)
    assert np.all(w > 0)
    assert np.sum(w) == pytest.approx(4 * math.pi, rel=1e-14)
    assert np.max(np.abs(rule_moment_errors(pts, w, degree))) < 1e-13
    # tight: some monomial of the next even degree is not integrated exactly
    assert np.max(np.abs(rule_moment_errors(pts, w, degree + 1))) > 1e-6
    sig, ws = antipodal_pairs(pts, w)
    assert len(sig) == M // 2
    assert 2 * np.sum(ws) == pytest.approx(4 * math.pi, rel=1e-14)


def test_icosahedron_is_equal_weight_and_regular():
    pts, w, _ = sphere_rule(12)
    np.testing.assert_allclose(w, 4 * math.pi / 12, rtol=1e-15)
    # every vertex has exactly five nearest neighbours at the same angle
    d = np.linalg.norm(pts[:, None] - pts[None], axis=-1)
    d[d == 0] = np.inf
    nearest = np.sort(d, axis=1)[:, :5]
    np.testing.assert_allclose(nearest, nearest[0, 0], rtol=1e-14)


def test_antipodal_pairs_rejects_non_antipodal_rule():
    pts = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    with pytest.raises(ValueError):
        antipodal_pairs(pts, np.ones(2))
