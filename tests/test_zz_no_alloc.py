"""dgfs_collide_noalloc: Q(f, f) without any device allocation.

Some callers cannot allocate device memory when they run (their memory is reserved up front,
or they must not pay the synchronisation an allocation can cause). dgfs_collide_noalloc serves
them: it evaluates the same operator as dgfs_collide but keeps its scratch in the library's fixed
64 MiB device array (with the dense circulant translate kernel for FP32/FP64 plans, where
dgfs_collide takes the translates in Fourier space). These tests call it through the C ABI, twice
in a row (the array keeps the previous call's contents), and compare each result with
dgfs_collide's on the same input.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1809_10186_gb300 import binding, workloads as W

pytestmark = pytest.mark.gpu

# relative L2 against dgfs_collide's result: the same kernels for F16S; for FP32 two translate
# methods, each within 1e-5 of the loss term of the FP64 oracle (Q itself is a few % of the loss)
TOL = {"fp32": 1e-4, "f16s": 1e-5, "fp64": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1809_10186_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def _noalloc(plan, f):
    out = torch.empty_like(f)
    st = binding.lib().dgfs_collide_noalloc(plan.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                            ctypes.c_int64(f.shape[0]), binding._stream_ptr())
    return st, out


@pytest.mark.parametrize("N,L,M,prec,B", [(16, 5.0, 12, "fp32", 5), (32, 7.0, 38, "fp32", 4),
                                          (32, 7.0, 38, "f16s", 4), (16, 5.0, 12, "fp64", 3)])
def test_noalloc_matches_collide_twice(N, L, M, prec, B):
    dt = torch.float64 if prec == "fp64" else torch.float32
    plan = binding.Plan(N=N, L=L, gamma=0.52, M=M, N_rho=N, precision=prec)
    for call in range(2):
        F, _ = W.two_maxwellian(B, N, L, 500 + 10 * N + call)
        f = torch.from_numpy(F).to("cuda", dt)
        st, q = _noalloc(plan, f)
        assert st == 0, binding.lib().dgfs_last_error_message().decode()
        ref = plan.collide(f)
        torch.cuda.synchronize()
        plan.stream_status()
        rel = (torch.linalg.norm(q - ref) / torch.linalg.norm(ref)).item()
        print(prec, N, call, "rel %.3g" % rel)
        assert rel < TOL[prec], (call, rel)


def test_noalloc_rejects_batches_beyond_the_fixed_array():
    N, L = 32, 7.0
    plan = binding.Plan(N=N, L=L, gamma=0.52, M=38, N_rho=N, precision="fp32")
    f = torch.zeros(64, N, N, N, device="cuda")
    st, _ = _noalloc(plan, f)
    assert st == 1
    msg = binding.lib().dgfs_last_error_message().decode()
    assert "exceeds" in msg and "fixed" in msg


def test_noalloc_rejects_fp64_beyond_n24():
    """FP64 plans at N = 32 run through dgfs_collide, not the fixed-scratch call."""
    plan = binding.Plan(N=32, L=7.0, gamma=0.52, M=38, N_rho=8, precision="fp64")
    f = torch.zeros(1, 32, 32, 32, dtype=torch.float64, device="cuda")
    st, _ = _noalloc(plan, f)
    assert st == 2
    assert "N <= 24" in binding.lib().dgfs_last_error_message().decode()
