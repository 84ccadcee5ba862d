"""The DG element collision term on the GPU (Sec. 3.4): the SVD variant (eqs.
eq_coln_derivation_SVD_3/4) evaluated by dgfs_dg_collide against the oracle's direct triple sum
(eq. HH), with truncation, chunking over elements and argument errors."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from oracle import dg as D
from paper_1809_10186_gb300 import binding, workloads as W

pytestmark = pytest.mark.gpu

# the nodal basis gives symmetric slices H[m], so every term is a quadratic Q(f_r, f_r): on the
# tensor cores for F16S (its tolerance), on the CUDA cores otherwise
TOL = {"fp64": 1e-10, "fp32": 1e-5, "f16s": 1e-3}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1809_10186_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def _elements(E, K, N, L, seed):
    """E elements of K nodal two-Maxwellian mixtures each (the slab workload's inputs)."""
    F, _ = W.two_maxwellian(E * K, N, L, seed)
    return F.reshape(E, K, N, N, N)


def _loss_part(op, H, F):
    K = H.shape[0]
    out = np.zeros_like(F)
    for m in range(K):
        for a in range(K):
            for b in range(K):
                out[m] += H[m, a, b] * np.real(O.loss_Q(op, F[a], F[b]))
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32", "f16s"])
def test_dg_svd_variant_matches_direct_sum(prec):
    N, L, gamma, M, K, E = 16, 5.0, 0.38, 12, 3, 3
    _, _, H = binding.host_dg_tensor(K)
    F = _elements(E, K, N, L, 31)
    dt = torch.float64 if prec == "fp64" else torch.float32
    if prec != "fp64":
        F = F.astype(np.float32).astype(np.float64)
    plan = binding.Plan(N=N, L=L, gamma=gamma, M=M, N_rho=N, precision=prec)
    dg = binding.DGElement(plan, H)
    assert dg.ranks == [u.shape[1] for u in D.svd_factors(H)[0]]
    C = dg.collide(torch.from_numpy(F).to("cuda", dt)).double().cpu().numpy()
    plan.stream_status()
    op = O.OraclePlan(N, L, gamma=gamma, M=M, Nrho=N, nyquist="sym")
    for e in range(E):
        ref = D.element_collision_direct(op, H, F[e])
        err = np.linalg.norm(C[e] - ref) / np.linalg.norm(_loss_part(op, H, F[e]))
        print(prec, "element", e, "ranks", dg.ranks, "err/|C-| %.3g" % err)
        assert err < TOL[prec]
    dg.close()
    plan.close()


def test_dg_non_symmetric_tensor_takes_the_bilinear_svd_form():
    """A tensor with non-symmetric slices (not a nodal-basis H) goes through the general SVD
    factors and bilinear Q(f_r, g_r); it must still equal the direct sum eq. HH."""
    N, L, K, E = 8, 3.5, 3, 2
    _, _, H = binding.host_dg_tensor(K)
    H = H.copy()
    H[:, 0, 1] += 0.05
    H[1, 2, 0] -= 0.03
    F = _elements(E, K, N, L, 51)
    plan = binding.Plan(N=N, L=L, gamma=0.3, M=12, N_rho=6, precision="fp64")
    dg = binding.DGElement(plan, H)
    C = dg.collide(torch.from_numpy(F).cuda()).cpu().numpy()
    plan.stream_status()
    op = O.OraclePlan(N, L, gamma=0.3, M=12, Nrho=6, nyquist="sym")
    for e in range(E):
        ref = D.element_collision_direct(op, H, F[e])
        assert np.linalg.norm(C[e] - ref) / np.linalg.norm(_loss_part(op, H, F[e])) < 1e-10
    dg.close()
    plan.close()


def test_dg_truncated_ranks_and_chunking():
    """svd_tol drops small singular values exactly as the oracle's truncation does; the result
    does not depend on how many elements one internal pass takes."""
    N, L, K, E = 16, 5.0, 4, 5
    _, _, H = binding.host_dg_tensor(K)
    F = _elements(E, K, N, L, 41)
    plan = binding.Plan(N=N, L=L, gamma=0.52, M=12, N_rho=N, precision="fp64")
    a = binding.DGElement(plan, H, svd_tol=0.15, max_elements=2)
    b = binding.DGElement(plan, H, svd_tol=0.15, max_elements=8)
    assert a.ranks == [u.shape[1] for u in D.svd_factors(H, 0.15)[0]]
    assert a.total_rank < K * K
    f = torch.from_numpy(F).cuda()
    ca, cb = a.collide(f), b.collide(f)
    plan.stream_status()
    assert torch.equal(ca, cb)
    op = O.OraclePlan(N, L, gamma=0.52, M=12, Nrho=N, nyquist="sym")
    ref = D.element_collision_svd(op, H, F[4], 0.15)
    err = np.linalg.norm(ca[4].cpu().numpy() - ref) / np.linalg.norm(_loss_part(op, H, F[4]))
    assert err < 1e-10
    a.close()
    b.close()
    plan.close()


def test_dg_argument_errors():
    N = 8
    plan = binding.Plan(N=N, L=3.0, gamma=0.0, M=6, N_rho=4, precision="fp32")
    _, _, H = binding.host_dg_tensor(3)
    lib = binding.lib()
    h = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    assert lib.dgfs_dg_create(plan.handle, 1, H.ctypes.data_as(dp), 0.0, 4, ctypes.byref(h)) == 1   # K < 2
    assert lib.dgfs_dg_create(plan.handle, 3, None, 0.0, 4, ctypes.byref(h)) == 1                    # NULL H
    assert lib.dgfs_dg_create(plan.handle, 3, H.ctypes.data_as(dp), 1.5, 4, ctypes.byref(h)) == 1   # svd_tol
    dg = binding.DGElement(plan, H)
    f = torch.zeros(2, 3, N, N, N, device="cuda")
    assert lib.dgfs_dg_collide(dg.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(f.data_ptr()), 2, None) == 1
    assert lib.dgfs_dg_collide(dg.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(0), 0, None) == 0   # E = 0
    dg.close()
    plan.close()
