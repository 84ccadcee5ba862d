"""The autotuner (dgfs_plan_autotune): radial points per CTA of the tensor-core kernels and nodes per
chunk, chosen by timing on the caller's batch and cached per shape."""
import numpy as np
import pytest
import torch

from paper_1809_10186_gb300 import binding, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1809_10186_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def _rule_rpc(prec, nodes, n_rho):
    """The batch-size rule of the tensor-core launchers: the most of 4, 2, 1 radial points per item that
    divides N_rho while the items (CTA pairs for the split-data kernels) fill the GPU 16 times over."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    per = 2 if prec in ("f16x3", "bf16x3") else 1
    for c in (4, 2):
        if n_rho % c == 0 and per * (n_rho // c) * nodes >= 16 * sms:
            return c
    return 1


def _time(plan, f, q, reps=3):
    plan.collide(f, out=q)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        plan.collide(f, out=q)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


@pytest.mark.parametrize("prec,B", [("f16s", 256), ("f16x3", 128), ("fp32", 64)])
def test_autotune_choice_is_never_slower_and_every_candidate_gives_the_same_result(prec, B):
    N, L = 32, 7.0
    F, _ = W.two_maxwellian(B, N, L, 2024, dtype=np.float32)
    f = torch.from_numpy(F).cuda()
    q = torch.empty_like(f)
    plan = binding.Plan(N=N, L=L, gamma=0.52, M=38, N_rho=N, svd_tol=1e-8, precision=prec, max_batch=B)
    ref = plan.collide(f).clone()
    # every configuration the tuner may pick computes the same arithmetic per radial point
    rpcs = (0, 1, 2, 4, 8) if prec != "fp32" else (0,)
    for rpc in rpcs:
        for chunk in (0, B // 2, B // 4):
            plan.set_tuning(rpc, chunk)
            out = plan.collide(f)
            plan.stream_status()
            assert torch.equal(out, ref), (rpc, chunk)
    plan.set_tuning(0, 0)
    t_default = min(_time(plan, f, q) for _ in range(2))
    rep = plan.autotune(f)
    print(prec, rep)
    assert rep["cached"] in (0, 1)
    if not rep["cached"]:
        assert rep["candidates"] == len(rpcs if prec != "fp32" else (0,)) * 3 or rep["candidates"] >= 3
    assert rep["ms_per_node_tuned"] <= rep["ms_per_node_default"] * 1.0001
    if prec != "fp32" and rep["ms_per_node_tuned"] == rep["ms_per_node_default"]:
        # the batch-size rule won: the report (and the plan) carry the rule's own value
        assert rep["rpc"] == _rule_rpc(prec, B, 32), rep
    t_tuned = min(_time(plan, f, q) for _ in range(2))
    print("%s B=%d default %.3f ms, tuned %.3f ms (rpc %d, chunk %d)" % (prec, B, t_default, t_tuned, rep["rpc"],
                                                                         rep["chunk_nodes"]))
    assert t_tuned <= 1.05 * t_default
    assert torch.equal(plan.collide(f), ref)
    plan.stream_status()
    # a second plan of the same shape takes the cached choice without timing
    again = binding.Plan(N=N, L=L, gamma=0.52, M=38, N_rho=N, svd_tol=1e-8, precision=prec, max_batch=B)
    rep2 = again.autotune(f)
    assert rep2["cached"] == 1 and rep2["rpc"] == rep["rpc"] and rep2["chunk_nodes"] == rep["chunk_nodes"]
    assert torch.equal(again.collide(f), ref)
    again.stream_status()
    plan.close()
    again.close()


def test_set_tuning_rejects_a_radial_split_that_does_not_divide_n_rho():
    plan = binding.Plan(N=16, L=5.0, gamma=0.52, M=12, N_rho=12, precision="f16s")
    with pytest.raises(binding.DGFSError):
        plan.set_tuning(5, 0)
    plan.close()


def test_plan_fingerprint_equals_the_host_builders():
    """dgfs_plan_fingerprint of a device plan equals dgfs_host_plan_fingerprint of its descriptor."""
    kw = dict(N=32, L=7.0, gamma=0.52, M=38, N_rho=32, svd_tol=1e-8, precision="f16s")
    plan = binding.Plan(max_batch=16, **kw)
    assert plan.fingerprint() == binding.host_plan_fingerprint(**kw)
    plan.close()
