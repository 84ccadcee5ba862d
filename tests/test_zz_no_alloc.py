"""dgfs_collide_noalloc: Q(f, f) without any device allocation.

Some callers cannot allocate device memory when they run (their memory is reserved up front,
or they must not pay the synchronisation an allocation can cause). dgfs_collide_noalloc serves
them: it evaluates the same operator as dgfs_collide but keeps its scratch in the library's fixed
64 MiB device array (with the dense circulant translate kernel for FP32/FP64 plans, where
dgfs_collide takes the translates in Fourier space). These tests call it through the C ABI, twice
in a row (the array keeps the previous call's contents), and compare each result with
dgfs_collide's on the same input and with the FP64 oracle.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_1809_10186_gb300 import binding, workloads as W

from oracle_refs import batch_errors

pytestmark = pytest.mark.gpu

# relative L2 against dgfs_collide's result: the same kernels for F16S; for FP32 two translate
# methods, each within 1e-5 of the loss term of the FP64 oracle (Q itself is a few % of the loss)
TOL = {"fp32": 1e-4, "f16s": 1e-5, "fp64": 1e-10}
# against the FP64 oracle, by ||Q|| and by ||Q-|| (batch errors): the tolerances of the parity tests
TOL_Q = {"fp64": 1e-10, "fp32": 1e-5, "f16s": 1e-2, "bf16s": 5e-2, "f16x3": 1e-5, "bf16x3": 1e-3}
TOL_L = {"fp64": 1e-10, "fp32": 1e-5, "f16s": 1e-3, "bf16s": 5e-3, "f16x3": 1e-5, "bf16x3": 1e-4}


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


@pytest.mark.parametrize("prec", ["fp32", "f16s", "bf16s", "f16x3", "bf16x3", "fp64"])
def test_noalloc_matches_the_oracle(prec):
    """The allocation-free call against the FP64 oracle itself (not only against dgfs_collide, which
    runs the same tensor-core kernels for the 16-bit plans), two calls in a row."""
    N, L, M, B = 16, 5.0, 12, 2
    dt = torch.float64 if prec == "fp64" else torch.float32
    plan = binding.Plan(N=N, L=L, gamma=0.52, M=M, N_rho=N, precision=prec)
    op = O.OraclePlan(N, L, gamma=0.52, M=M, Nrho=N, nyquist="sym")
    for call in range(2):
        F, _ = W.two_maxwellian(B, N, L, 640 + call, dtype=np.float64 if prec == "fp64" else np.float32)
        st, q = _noalloc(plan, torch.from_numpy(F).to("cuda", dt))
        assert st == 0, binding.lib().dgfs_last_error_message().decode()
        torch.cuda.synchronize()
        plan.stream_status()
        Fd = F.astype(np.float64)
        e = batch_errors(list(q.double().cpu().numpy()), [O.fast_Q(op, Fd[i]) for i in range(B)],
                         [np.real(O.loss_Q(op, Fd[i], Fd[i])) for i in range(B)])
        print(prec, call, e)
        assert e["batch_q"] < TOL_Q[prec] and e["batch_loss"] < TOL_L[prec], e


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
