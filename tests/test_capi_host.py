"""The C-ABI library loads, exports every declared symbol, and its host-only plan builder
agrees with the oracle's independent quadrature and translate operator (no GPU)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1809_10186_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1809_10186_gb300 import build
    build.build()
    return binding.lib()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "dgfs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dgfs_\w+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        assert n in binding._SIGNATURES, "binding misses " + n


@pytest.mark.parametrize("N", [8, 16, 32])
def test_gauss_legendre_matches_oracle(lib, N):
    cr, wr, _, R, _ = binding.host_quadrature(N=N, L=7.0, M=6, N_rho=N)
    x, w = O.gauss_legendre(N, 0.0, R)
    assert R == pytest.approx(4 * 7.0 / (3 + math.sqrt(2)), rel=1e-15)
    np.testing.assert_allclose(cr, x, rtol=0, atol=1e-13)
    np.testing.assert_allclose(wr, w, rtol=1e-12)


@pytest.mark.parametrize("M", [6, 12, 26, 38])
def test_sphere_rules_match_oracle(lib, M):
    _, _, sig, _, _ = binding.host_quadrature(N=8, L=3.0, M=M)
    pts, wts, _ = O.sphere_rule(M)
    assert sig.shape == (M // 2, 4)
    # same point set (as antipodal pairs) with the same weights
    full = np.concatenate([sig[:, :3], -sig[:, :3]])
    fw = np.concatenate([sig[:, 3], sig[:, 3]])
    for p, w in zip(pts, wts):
        d = np.linalg.norm(full - p, axis=1)
        i = int(np.argmin(d))
        assert d[i] < 1e-12 and abs(fw[i] - w) < 1e-12


def test_default_kernel_constant(lib):
    omega = 0.74
    _, _, _, _, b = binding.host_quadrature(N=8, L=3.0, M=6, gamma=2 * (1 - omega))
    assert b == pytest.approx(O.b_vhs(omega), rel=1e-14)


@pytest.mark.parametrize("N", [8, 16])
def test_translate_filter_is_oracle_translate(lib, N):
    """The circulant filter applied to a grid function equals the oracle's symmetric translate."""
    L = 4.0
    plan = O.OraclePlan(N, L, M=6, Nrho=2, nyquist="sym")
    rng = np.random.default_rng(1)
    f = rng.random((N, N, N))
    s = np.array([0.731, -1.27, 2.91])
    mats = []
    for a in range(3):
        filt = binding.host_translate_filter(N, L, s[a])
        mats.append(np.array([[filt[(i - j) % N] for j in range(N)] for i in range(N)]))
    got = np.einsum("ai,bj,ck,ijk->abc", mats[0], mats[1], mats[2], f)
    np.testing.assert_allclose(got, plan.translate_hat(plan.dft3(f), s), atol=1e-12)


def test_invalid_descriptors_rejected_before_any_cuda_call(lib):
    for kw, frag in (({"N": 7}, "N must be"), ({"N": 20}, "N must be"), ({"L": -1.0}, "L must"),
                     ({"M": 10}, "sphere rule"), ({"N_rho": 100}, "N_rho")):
        d, _ = binding.make_desc(**{"N": 8, "L": 3.0, "M": 6, **kw})
        h = ctypes.c_void_p()
        st = lib.dgfs_plan_create(ctypes.byref(d), ctypes.byref(h))
        assert st == 1 and not h.value, kw
        assert frag in lib.dgfs_last_error_message().decode()
    # a user sphere rule that is not normalised
    d, keep = binding.make_desc(N=8, L=3.0, sphere=np.array([[1.0, 0, 0, 1.0], [0, 1.0, 0, 1.0]]))
    assert lib.dgfs_plan_create(ctypes.byref(d), ctypes.byref(ctypes.c_void_p())) == 1


def test_null_and_destroyed_plans_rejected(lib):
    assert lib.dgfs_collide(None, None, None, 1, None) == 7
    assert lib.dgfs_plan_destroy(None) == 0
    assert lib.dgfs_plan_create(None, None) == 1


@pytest.mark.parametrize("K", [2, 3, 4, 6, 9])
def test_dg_tensor_matches_oracle(lib, K):
    """Gauss-Lobatto nodes, mass matrix and H of the C library against the oracle's own
    construction (Sec. 3.4, eqs. eq_massMatrix and eq_stiffMatrix3)."""
    from oracle import dg as D
    nodes, M, H = binding.host_dg_tensor(K)
    on, oM, oH = D.dg_tensors(K)
    np.testing.assert_allclose(nodes, on, atol=1e-14)
    np.testing.assert_allclose(M, oM, atol=1e-14)
    np.testing.assert_allclose(H, oH, atol=1e-14)


def test_dg_tensor_rejects_bad_K(lib):
    d = ctypes.POINTER(ctypes.c_double)
    buf = np.zeros(20 * 20 * 20)
    for K in (1, 17):
        assert lib.dgfs_host_dg_tensor(K, buf.ctypes.data_as(d), buf.ctypes.data_as(d), buf.ctypes.data_as(d)) == 1


# ---- VSS kernel (alpha != 1): the plan builder's tables against the oracle --------------------

@pytest.mark.parametrize("alpha", [1.0, 1.3, 1.5, 2.0])
def test_vss_factor_matches_oracle_quadrature(lib, alpha):
    """The library evaluates F(k, c_r, sigma) of eq. realGG as a Funk-Hecke series; the oracle by
    Gauss-Jacobi and Bessel quadrature about sigma."""
    from oracle import vss as V
    rng = np.random.default_rng(5)
    k = np.concatenate([[0.0, 1.0, 3.0], rng.uniform(0, 56, 60)])
    mu = rng.uniform(-1, 1, len(k))
    cr = rng.uniform(0, 6.6, len(k))
    got = binding.host_vss_factor(7.0, 0.38, alpha, k, mu, cr)
    b = V.b_vss(1 - 0.19, alpha)
    ref = np.array([V.F_vss(b, 0.38, alpha, 7.0, np.array([a]), np.array([m]), c)[0] for a, m, c in zip(k, mu, cr)])
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("N,loss,alpha", [(8, "paper", 1.5), (8, "conservative", 1.3), (12, "paper", 1.8)])
def test_vss_tables_match_oracle(lib, N, loss, alpha):
    """A = w_r w_p F(k, c_r, sigma_p) on the lattice (Nyquist modes at their own signed index) and
    the loss weight; the library's sphere pairs are matched to the oracle's up to order and sign."""
    from oracle import vss as V
    kw = dict(N=N, L=4.0, gamma=0.5, alpha=alpha, M=12, N_rho=6, loss=loss)
    A, GL = binding.host_vss_tables(**kw)
    _, _, sig, _, _ = binding.host_quadrature(**kw)
    pl = V.VSSPlan(N, 4.0, gamma=0.5, alpha=alpha, M=12, Nrho=6, nyquist="sym", loss=loss)
    Ao = np.fft.ifftshift(pl.A * pl.wsig[None, :, None, None, None], axes=(2, 3, 4))
    for p in range(sig.shape[0]):
        q = int(np.argmax(np.abs(pl.sigma @ sig[p, :3])))
        assert abs(abs(pl.sigma[q] @ sig[p, :3]) - 1) < 1e-12
        assert np.abs(A[:, p] - Ao[:, q]).max() < 1e-12 * np.abs(Ao).max()
    assert np.abs(GL - np.fft.ifftshift(pl.Gloss)).max() < 1e-12 * np.abs(pl.Gloss).max()


def test_vss_descriptors_rejected(lib):
    with pytest.raises(binding.DGFSError):
        binding.host_vss_tables(N=8, L=4.0, alpha=2.5, M=12)
    with pytest.raises(binding.DGFSError):
        binding.host_vss_tables(N=8, L=4.0, alpha=1.5, M=12, svd_tol=1e-3)
    with pytest.raises(binding.DGFSError):
        binding.host_vss_tables(N=8, L=4.0, alpha=1.0, M=12)
    with pytest.raises(binding.DGFSError):
        binding.host_vss_factor(4.0, 0.0, 1.5, [1.0], [1.5], [1.0])
    _, _, _, _, b = binding.host_quadrature(N=8, L=4.0, M=12, gamma=0.5, alpha=1.5)
    from oracle import vss as V
    assert b == pytest.approx(V.b_vss(0.75, 1.5), rel=1e-14)


@pytest.mark.parametrize("K", [2, 3, 4, 6])
def test_dg_stiffness_matches_oracle(lib, K):
    from oracle import slab as SL
    from oracle.dg import dg_tensors
    S, Minv = binding.host_dg_stiffness(K)
    np.testing.assert_allclose(S, SL.stiffness(K), atol=1e-13)
    np.testing.assert_allclose(Minv, np.linalg.inv(dg_tensors(K)[1]), rtol=1e-11, atol=1e-11)
    with pytest.raises(binding.DGFSError):
        binding.host_dg_stiffness(1)


def test_plan_fingerprint_tracks_every_input(lib):
    """dgfs_host_plan_fingerprint: a pure function of the descriptor (the same descriptor twice gives
    the same value); any change of a parameter that enters the tables (gamma, N_rho, the sphere rule,
    the SVD truncation) or of the precision changes it."""
    base = dict(N=16, L=5.0, gamma=0.52, M=12, N_rho=12, svd_tol=1e-8, precision="f16s")
    f0 = binding.host_plan_fingerprint(**base)
    assert f0 == binding.host_plan_fingerprint(**base)
    for change in (dict(gamma=0.53), dict(N_rho=16), dict(M=26), dict(svd_tol=1e-6), dict(precision="fp32"),
                   dict(L=5.5), dict(N=24)):
        other = dict(base, **change)
        assert binding.host_plan_fingerprint(**other) != f0, change


@pytest.mark.parametrize("B,chunk", [(2048, 2048), (2048, 1024), (3, 1), (5, 2), (5, 7), (9, 4096), (37, 4),
                                     (300, 64), (2, 4096), (1, 4096), (100000, 2048), (9216, 2048), (167, 10 ** 6)])
def test_host_pipeline_schedule_covers_the_batch(B, chunk):
    """dgfs_host_pipeline_schedule (the sub-batches of dgfs_collide_host): sizes in [1, chunk / 2]
    (1 for a one-node chunk) that sum to B; it starts at ceil(B / 32) when that is below the staging
    half (else the batch is split evenly) and grows by 4 while ramping up, the same steps mirrored at
    the end, and no sub-batch is more
    than 8 times its predecessor (its input copy hides behind the predecessor's compute)."""
    sizes = binding.host_pipeline_schedule(B, chunk)
    H = chunk // 2 if chunk >= 2 else 1
    assert sum(sizes) == B
    assert all(1 <= s <= H for s in sizes), sizes
    r0 = max(1, -(-B // 32))
    if r0 < H and 2 * r0 <= B:   # a ramp: it starts at ceil(B / 32)
        assert sizes[0] == r0, sizes
    else:                        # none: the batch split evenly into sub-batches of at most H
        assert max(sizes) - min(sizes) <= 1, sizes
    k = 0   # ramp steps: while the next size is 4 times the previous
    while k + 1 < len(sizes) and sizes[k + 1] == 4 * sizes[k]:
        k += 1
    assert sizes[:k] == sizes[::-1][:k], sizes
    assert all(b <= 8 * a for a, b in zip(sizes, sizes[1:])), sizes


def test_host_pipeline_schedule_of_the_headline_batch_and_errors():
    assert binding.host_pipeline_schedule(2048, 2048) == [64, 256, 704, 704, 256, 64]
    assert binding.host_pipeline_schedule(0, 16) == []
    with pytest.raises(binding.DGFSError):
        binding.host_pipeline_schedule(-1, 16)
    with pytest.raises(binding.DGFSError):
        binding.host_pipeline_schedule(8, 0)


def _handle_calls():
    """Every declared call that takes a plan, DG operator, slab or ragged schedule, with a NULL
    handle (or an empty plan list) and otherwise well-formed arguments."""
    n, i, d, q = ctypes.c_void_p(None), ctypes.c_int, ctypes.c_double, ctypes.c_int64
    return {
        "dgfs_plan_info": (n, n),
        "dgfs_collide": (n, n, n, q(1), n),
        "dgfs_collide2": (n, n, n, n, q(1), n),
        "dgfs_collide_jvp": (n, n, n, n, q(1), n),
        "dgfs_collide_vjp": (n, n, n, n, q(1), n),
        "dgfs_collide_dgamma": (n, n, n, q(1), n),
        "dgfs_collide_host": (n, n, n, q(1), n),
        "dgfs_collide_noalloc": (n, n, n, q(1), n),
        "dgfs_collide_ragged": (n, i(0), n, n, n, n, q(1), n, n, n),
        "dgfs_ragged_create": (n, i(0), n, n, n, n, q(1), n),
        "dgfs_ragged_collide": (n, n, n, n),
        "dgfs_slab_create": (n, i(3), i(2), n, d(1.0), n, n, d(0.0), n),
        "dgfs_slab_set_walls": (n, n, n),
        "dgfs_slab_rhs": (n, n, n, n),
        "dgfs_slab_ssprk": (n, i(2), n, d(0.01), i(2), n),
        "dgfs_stream_status": (n, n),
        "dgfs_ssprk": (n, i(2), n, q(1), d(0.01), d(1.0), i(1), n),
        "dgfs_moments": (n, n, n, q(1), n),
        "dgfs_dg_create": (n, i(3), n, d(0.0), q(1), n),
        "dgfs_dg_info": (n, n, n),
        "dgfs_dg_collide": (n, n, n, q(1), n),
        "dgfs_debug_inject": (n, i(0)),
        "dgfs_profile_begin": (n,),
        "dgfs_profile_end": (n, n),
        "dgfs_plan_autotune": (n, n, q(1), n, n),
        "dgfs_plan_set_tuning": (n, i(0), q(0)),
        "dgfs_plan_fingerprint": (n, n),
    }


def test_every_handle_call_rejects_a_null_handle_before_cuda(lib):
    """Argument and state errors return before any CUDA call: on a machine without a GPU a call
    that reached CUDA would answer DGFS_ERR_CUDA (4); these answer DGFS_ERR_INVALID_ARG (1) or
    DGFS_ERR_STATE (7) with a message. The list is checked against the header, so a new call that
    takes a handle must be added here."""
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "dgfs.h")).read(), flags=re.S)
    takes_handle = {m.group(1) for m in re.finditer(
        r"\b(dgfs_\w+)\s*\(\s*(?:const\s+)?dgfs_(?:plan|dg|slab|ragged)_t\b", src)}
    destroys = {f for f in takes_handle if f.endswith("_destroy")}
    calls = _handle_calls()
    assert takes_handle - destroys == set(calls)
    raw = ctypes.CDLL(lib._name)   # a separate handle: no argument conversions of the binding
    raw.dgfs_last_error_message.restype = ctypes.c_char_p
    for name, args in calls.items():
        st = getattr(raw, name)(*args)
        assert st in (1, 7), (name, st)
        assert raw.dgfs_last_error_message(), name
    for name in destroys:   # destroying NULL is a no-op
        assert getattr(raw, name)(ctypes.c_void_p(None)) == 0, name
