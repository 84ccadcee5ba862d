"""Quadrature rules of the FP64 CPU oracle.

TEST INFRASTRUCTURE. Only tests/, the smoke check and bench.py's CPU-baseline leg
may import this module; the GPU product path has its own, independent plan builder.

* Radial rule: Gauss-Legendre on [0, R] (Appendix, after eq. lowrank1: the radial
  integral over c_r uses Gauss-Legendre points). Built here by the Golub-Welsch method:
  the nodes are the eigenvalues of the symmetric tridiagonal Jacobi matrix of the
  Legendre recurrence and the weights come from the first eigenvector components.
* Sphere rule: the paper integrates over the (half) sphere with a symmetric quadrature
  (Appendix: spherical designs, M << N^2 points). The rules here are antipodal
  full-sphere rules derived from the mathematics, never copied from a table:
    M = 6   octahedron vertices, equal weights (exact to degree 3),
    M = 12  icosahedron vertices, equal weights (exact to degree 5); its 6 antipodal
            pairs form the 6-point half-sphere design that the BKW table uses,
    M = 26  octahedral orbits 6 + 12 + 8, weights fitted to the exact monomial moments
            up to degree 7,
    M = 38  octahedral orbits 6 + 8 + 24 (points (+-p, +-q, 0) and permutations, one free
            parameter p), p and the weights fitted to the moments up to degree 9.
  Exactness is verified against the closed-form monomial integrals below.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

FOUR_PI = 4.0 * math.pi


def gauss_legendre(n: int, a: float = -1.0, b: float = 1.0):
    """n-point Gauss-Legendre rule on [a, b] (Golub-Welsch). Returns (nodes, weights)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    if n == 1:
        x = np.zeros(1)
        w = np.full(1, 2.0)
    else:
        j = np.arange(1, n, dtype=np.float64)
        beta = j / np.sqrt(4.0 * j * j - 1.0)
        jac = np.diag(beta, 1) + np.diag(beta, -1)
        x, vec = np.linalg.eigh(jac)
        w = 2.0 * vec[0, :] ** 2
    half = 0.5 * (b - a)
    return half * x + 0.5 * (b + a), half * w


def sphere_monomial_integral(a: int, b: int, c: int) -> float:
    """Exact integral of x^a y^b z^c over the unit sphere S^2.

    Zero unless a, b, c are all even; otherwise
    2 Gamma((a+1)/2) Gamma((b+1)/2) Gamma((c+1)/2) / Gamma((a+b+c+3)/2).
    """
    if a % 2 or b % 2 or c % 2:
        return 0.0
    g = math.gamma
    return 2.0 * g((a + 1) / 2) * g((b + 1) / 2) * g((c + 1) / 2) / g((a + b + c + 3) / 2)


def _signed_permutations(v):
    pts = set()
    for perm in itertools.permutations(v):
        for signs in itertools.product((1.0, -1.0), repeat=3):
            pts.add(tuple(float(s * x) + 0.0 for s, x in zip(signs, perm)))
    return np.array(sorted(pts), dtype=np.float64)


def _orbit_vertices():          # (+-1, 0, 0): 6 points
    return _signed_permutations((1.0, 0.0, 0.0))


def _orbit_edges():             # (+-1, +-1, 0)/sqrt 2: 12 points
    s = 1.0 / math.sqrt(2.0)
    return _signed_permutations((s, s, 0.0))


def _orbit_corners():           # (+-1, +-1, +-1)/sqrt 3: 8 points
    s = 1.0 / math.sqrt(3.0)
    return _signed_permutations((s, s, s))


def _orbit_pq0(p: float):       # (+-p, +-q, 0) and permutations, p^2 + q^2 = 1: 24 points
    return _signed_permutations((p, math.sqrt(1.0 - p * p), 0.0))


def _icosahedron():
    phi = 0.5 * (1.0 + math.sqrt(5.0))
    base = []
    for s1 in (1.0, -1.0):
        for s2 in (1.0, -1.0):
            v = (0.0, s1 * 1.0, s2 * phi)
            base += [v, (v[1], v[2], v[0]), (v[2], v[0], v[1])]
    pts = np.array(base, dtype=np.float64)
    return pts / np.linalg.norm(pts, axis=1, keepdims=True)


def _monomials(degree: int):
    return [(a, b, c) for a in range(degree + 1) for b in range(degree + 1 - a)
            for c in range(degree + 1 - a - b)]


def rule_moment_errors(points, weights, degree: int) -> np.ndarray:
    """Rule minus exact integral for every monomial x^a y^b z^c with a+b+c <= degree."""
    out = []
    for a, b, c in _monomials(degree):
        val = np.sum(weights * points[:, 0] ** a * points[:, 1] ** b * points[:, 2] ** c)
        out.append(val - sphere_monomial_integral(a, b, c))
    return np.array(out)


def _fit_orbit_weights(orbits, degree):
    """One weight per orbit so that the rule matches the monomial moments up to `degree`."""
    mons = _monomials(degree)
    a_mat = np.zeros((len(mons), len(orbits)))
    rhs = np.zeros(len(mons))
    for i, (a, b, c) in enumerate(mons):
        rhs[i] = sphere_monomial_integral(a, b, c)
        for j, pts in enumerate(orbits):
            a_mat[i, j] = np.sum(pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
    w, *_ = np.linalg.lstsq(a_mat, rhs, rcond=None)
    resid = float(np.max(np.abs(a_mat @ w - rhs)))
    return w, resid


def _rule_from_orbits(orbits, orbit_weights):
    pts = np.concatenate(orbits, axis=0)
    wts = np.concatenate([np.full(len(o), w) for o, w in zip(orbits, orbit_weights)])
    return pts, wts


def sphere_rule(M: int):
    """Built-in antipodal full-sphere rule with M points. Returns (points[M,3], weights[M], degree)."""
    if M == 6:
        pts = _orbit_vertices()
        return pts, np.full(6, FOUR_PI / 6), 3
    if M == 12:
        pts = _icosahedron()
        return pts, np.full(12, FOUR_PI / 12), 5
    if M == 26:
        orbits = [_orbit_vertices(), _orbit_edges(), _orbit_corners()]
        w, resid = _fit_orbit_weights(orbits, 7)
        if resid > 1e-13 or np.any(w <= 0):
            raise RuntimeError("26-point rule: moment fit failed")
        pts, wts = _rule_from_orbits(orbits, w)
        return pts, wts, 7
    if M == 38:
        def resid_at(p):
            orbits = [_orbit_vertices(), _orbit_corners(), _orbit_pq0(p)]
            return _fit_orbit_weights(orbits, 9)[1]
        # golden-section search of the moment residual over p in (0, 1/sqrt 2)
        lo, hi = 0.05, 1.0 / math.sqrt(2.0) - 1e-6
        grid = np.linspace(lo, hi, 400)
        vals = [resid_at(p) for p in grid]
        i = int(np.argmin(vals))
        lo, hi = grid[max(i - 1, 0)], grid[min(i + 1, len(grid) - 1)]
        g = 0.5 * (math.sqrt(5.0) - 1.0)
        x1, x2 = hi - g * (hi - lo), lo + g * (hi - lo)
        f1, f2 = resid_at(x1), resid_at(x2)
        for _ in range(200):
            if f1 < f2:
                hi, x2, f2 = x2, x1, f1
                x1 = hi - g * (hi - lo)
                f1 = resid_at(x1)
            else:
                lo, x1, f1 = x1, x2, f2
                x2 = lo + g * (hi - lo)
                f2 = resid_at(x2)
            if hi - lo < 1e-16:
                break
        p = 0.5 * (lo + hi)
        orbits = [_orbit_vertices(), _orbit_corners(), _orbit_pq0(p)]
        w, resid = _fit_orbit_weights(orbits, 9)
        if resid > 1e-12 or np.any(w <= 0):
            raise RuntimeError("38-point rule: moment fit failed (resid %g)" % resid)
        pts, wts = _rule_from_orbits(orbits, w)
        return pts, wts, 9
    raise ValueError("no built-in sphere rule with M=%d points (have 6, 12, 26, 38)" % M)


def product_rule(n_z: int, n_phi: int):
    """Antipodal product rule: Gauss-Legendre in z = cos(theta), n_phi (even) equal phi steps."""
    if n_phi % 2:
        raise ValueError("n_phi must be even for an antipodal rule")
    z, wz = gauss_legendre(n_z, -1.0, 1.0)
    z = 0.5 * (z - z[::-1])                 # exact symmetry of the nodes
    wz = 0.5 * (wz + wz[::-1])
    phi = (np.arange(n_phi) + 0.5) * 2.0 * math.pi / n_phi
    Z, P = np.meshgrid(z, phi, indexing="ij")
    s = np.sqrt(1.0 - Z * Z)
    pts = np.stack([s * np.cos(P), s * np.sin(P), Z], -1).reshape(-1, 3)
    w = (wz[:, None] * np.full(n_phi, 2.0 * math.pi / n_phi)[None, :]).ravel()
    return pts, w


def antipodal_pairs(points, weights):
    """Split an antipodal rule into one representative per pair {sigma, -sigma}.

    Returns (sigma[M/2, 3], w[M/2]) where w is the weight of EACH of the two points.
    Raises if the rule is not antipodally symmetric with equal pair weights.
    """
    points = np.asarray(points, dtype=np.float64)
    weights = np.asarray(weights, dtype=np.float64)
    used = np.zeros(len(points), dtype=bool)
    reps, wts = [], []
    for i in range(len(points)):
        if used[i]:
            continue
        d = np.linalg.norm(points + points[i], axis=1)
        j = int(np.argmin(d))
        if d[j] > 1e-12 or used[j] or j == i or abs(weights[i] - weights[j]) > 1e-12 * abs(weights[i]):
            raise ValueError("sphere rule is not antipodal")
        used[i] = used[j] = True
        reps.append(points[i])
        wts.append(weights[i])
    return np.array(reps), np.array(wts)
