"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random parameters and evaluates distribution functions on the
velocity grid; it contains none of the collision operator's arithmetic. Both the CUDA
path (through tests and bench.py) and the CPU oracle receive the arrays it returns.

Random numbers come from numpy's Philox counter-based generator, so a seed gives the
same stream on every platform.

Workloads (nondimensional units of Sec. 2.1):
  * bkw:            Bobylev-Krook-Wu distribution at time t (Sec. 4.3, eq. bkw_f).
  * two_maxwellian: per node a sum of two Maxwellians n (pi T)^{-3/2} exp(-|c-u|^2 / T)
                    (the Maxwellian of Sec. 3.5) with n ~ U[0.5, 1.5],
                    u ~ N(0, 0.3^2) per component, T ~ U[0.7, 1.3].
  * near_equilibrium: one Maxwellian per node, n ~ U[0.8, 1.2], T ~ U[1, 2],
                    |u| ~ U[0, 0.5] in a uniformly random direction, times (1 + 0.01 xi)
                    with xi standard normal per grid point (a cavity-like state with a
                    wall-temperature ratio up to 2).
  * directions:     standard normal fields scaled to unit Euclidean norm per node.
  * rough:          uniform [0, 1) values per grid point (carries Nyquist content).
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 1809


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def velocity_grid(N: int, L: float) -> np.ndarray:
    """Cell centres -L + (j + 1/2) 2L/N, j = 0..N-1 (one axis)."""
    return -L + (np.arange(N, dtype=np.float64) + 0.5) * (2.0 * L / N)


def _c2_and_axes(N, L):
    c = velocity_grid(N, L)
    cx, cy, cz = np.meshgrid(c, c, c, indexing="ij")
    return cx, cy, cz


def maxwellian(N, L, n, u, T):
    cx, cy, cz = _c2_and_axes(N, L)
    d2 = (cx - u[0]) ** 2 + (cy - u[1]) ** 2 + (cz - u[2]) ** 2
    return n / (math.pi * T) ** 1.5 * np.exp(-d2 / T)


def bkw(N, L, t):
    """f(t, c) for the constant kernel B = 1/(4 pi); valid for t > 6 ln 2.5."""
    cx, cy, cz = _c2_and_axes(N, L)
    c2 = cx * cx + cy * cy + cz * cz
    K = 1.0 - math.exp(-t / 6.0)
    return (np.exp(-c2 / (2 * K)) / (2 * (2 * math.pi * K) ** 1.5)
            * ((5 * K - 3) / K + (1 - K) / K ** 2 * c2))


def two_maxwellian(B, N, L, seed, dtype=np.float64):
    g = rng(seed)
    out = np.empty((B, N, N, N), dtype=dtype)
    params = []
    for b in range(B):
        f = np.zeros((N, N, N))
        p = []
        for _ in range(2):
            n = g.uniform(0.5, 1.5)
            u = g.normal(0.0, 0.3, size=3)
            T = g.uniform(0.7, 1.3)
            f += maxwellian(N, L, n, u, T)
            p.append((n, u, T))
        out[b] = f
        params.append(p)
    return out, params


def near_equilibrium(B, N, L, seed, dtype=np.float64):
    g = rng(seed)
    out = np.empty((B, N, N, N), dtype=dtype)
    for b in range(B):
        n = g.uniform(0.8, 1.2)
        T = g.uniform(1.0, 2.0)
        speed = g.uniform(0.0, 0.5)
        d = g.normal(size=3)
        d /= np.linalg.norm(d)
        f = maxwellian(N, L, n, speed * d, T)
        out[b] = f * (1.0 + 0.01 * g.normal(size=f.shape))
    return out


def directions(B, N, seed, dtype=np.float64):
    g = rng(seed)
    v = g.normal(size=(B, N, N, N))
    v /= np.sqrt(np.sum(v * v, axis=(1, 2, 3), keepdims=True))
    return v.astype(dtype)


def rough(B, N, seed, dtype=np.float64):
    return rng(seed).random((B, N, N, N)).astype(dtype)


# ---- the five workload configurations --------------------------------------------------

def omega_to_gamma(omega):
    """VHS exponent of |c - c_*| in B: gamma = 2 (1 - omega) (eq. B_gen)."""
    return 2.0 * (1.0 - omega)


CONFIGS = {
    # single node, Maxwell molecules, BKW initial datum, FP64
    "bkw_n16": dict(N=16, L=8.0, Nrho=16, M=6, gamma=0.0, b=1.0 / (4.0 * math.pi),
                    R=2.0 * 8.0 * math.sqrt(2.0) / (3.0 + math.sqrt(2.0)), B=1, prec="fp64",
                    seed=SEED_BASE + 1),
    # 1-D slab: 16 elements x 3 nodes, argon VHS omega = 0.81, FP32
    "slab_n24": dict(N=24, L=6.0, Nrho=24, M=12, gamma=omega_to_gamma(0.81), B=48,
                     prec="fp32", seed=SEED_BASE + 2),
    # primary workload: 2048 nodes, omega = 0.74, N = 32, M = 38, SVD at 1e-8
    "vhs_n32": dict(N=32, L=7.0, Nrho=32, M=38, gamma=omega_to_gamma(0.74), B=2048,
                    svd_tol=1e-8, prec="bf16x3", seed=SEED_BASE + 3),
    # ragged cavity mesh: 32 x 32 quads x 9 nodes, N in {16, 24, 32} (40/40/20 %)
    "cavity_ragged": dict(Ns=(16, 24, 32), split=(0.4, 0.4, 0.2), L=9.0, M=26,
                          omegas=(0.5, 0.74, 0.81), B=9216, seed=SEED_BASE + 4),
    # differentiation: 512 nodes, N = 32, omega = 0.81, FP32
    "grad_n32": dict(N=32, L=7.0, Nrho=32, M=38, gamma=omega_to_gamma(0.81), B=512,
                     prec="fp32", seed=SEED_BASE + 5),
    # 1-D Fourier heat transfer (Sec. 4.4 setup): argon, Maxwell molecules (omega = 1), walls at
    # 263 K and 283 K (T_ref = 273 K) at rest, Kn (Cercignani) = 1.582, i.e. Kn (eq. Kn) = 1.582 * 2 / pi;
    # 10 elements of K = 3 Gauss-Lobatto nodes, N = 24 on [-5.09, 5.09]^3, M = 12 (6 on the half sphere)
    "fourier_slab": dict(N=24, L=5.09, Nrho=24, M=12, gamma=0.0, K=3, I=10, Kn=1.582 * 2.0 / math.pi,
                         T_left=263.0 / 273.0, T_right=283.0 / 273.0, dt=0.002, prec="fp32"),
    # VSS kernel (eq. B_gen, alpha != 1): argon's VSS parameters omega = 0.81, alpha = 1.40,
    # 256 nodes, N = 32, M = 38, FP32 (one transform per radial and sphere point)
    "vss_n32": dict(N=32, L=7.0, Nrho=32, M=38, gamma=omega_to_gamma(0.81), alpha=1.40, B=256,
                    prec="fp32", seed=SEED_BASE + 6),
}


def ragged_layout(B, Ns, split, omegas, seed):
    """Per-node grid size and VHS omega for the ragged mesh, in a seeded random order."""
    g = rng(seed)
    counts = [int(round(B * s)) for s in split]
    counts[-1] = B - sum(counts[:-1])
    node_N = np.concatenate([np.full(c, n) for c, n in zip(counts, Ns)])
    node_N = node_N[g.permutation(B)]
    node_omega = np.asarray(omegas)[g.integers(0, len(omegas), size=B)]
    return node_N.astype(np.int32), node_omega
