"""Thin Python binding of the C ABI in include/dgfs.h (argument marshalling only).

Every computation runs in libdgfs.so; this module passes device pointers, sizes and the
current CUDA stream. It raises if the library has not been built: there is no fallback.

    from paper_1809_10186_gb300.binding import Plan
    plan = Plan(N=32, L=7.0, gamma=0.52, M=38, N_rho=32, svd_tol=1e-8, precision="fp32")
    Q = plan.collide(f)            # f: CUDA tensor [B, N, N, N], float32 (float64 for fp64)
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libdgfs.so")

PRECISIONS = {"fp64": 0, "fp32": 1, "f16s": 2, "bf16s": 3, "f16x3": 4, "bf16x3": 5}
LOSS_MODES = {"paper": 0, "conservative": 1}
STATUS = {0: "DGFS_OK", 1: "DGFS_ERR_INVALID_ARG", 2: "DGFS_ERR_UNSUPPORTED", 3: "DGFS_ERR_OOM",
          4: "DGFS_ERR_CUDA", 5: "DGFS_ERR_TIMEOUT", 6: "DGFS_ERR_NUMERIC", 7: "DGFS_ERR_STATE"}


class dgfs_plan_desc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("L", ctypes.c_double), ("R", ctypes.c_double),
                ("gamma", ctypes.c_double), ("b", ctypes.c_double), ("M", ctypes.c_int),
                ("sphere_xyzw", ctypes.POINTER(ctypes.c_double)), ("N_rho", ctypes.c_int),
                ("svd_tol", ctypes.c_double), ("svd_rank", ctypes.c_int),
                ("precision", ctypes.c_int), ("loss_mode", ctypes.c_int),
                ("max_batch", ctypes.c_int64), ("alpha", ctypes.c_double)]


class dgfs_plan_info_t(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("N_rho", ctypes.c_int), ("n_pairs", ctypes.c_int),
                ("svd_rank_used", ctypes.c_int), ("precision", ctypes.c_int),
                ("loss_mode", ctypes.c_int), ("L", ctypes.c_double), ("R", ctypes.c_double),
                ("gamma", ctypes.c_double), ("b", ctypes.c_double),
                ("chunk_nodes", ctypes.c_int64), ("workspace_bytes", ctypes.c_size_t),
                ("table_bytes", ctypes.c_size_t), ("alpha", ctypes.c_double)]


class dgfs_tune_report(ctypes.Structure):
    _fields_ = [("rpc", ctypes.c_int), ("chunk_nodes", ctypes.c_int64), ("ms_per_node_default", ctypes.c_double),
                ("ms_per_node_tuned", ctypes.c_double), ("candidates", ctypes.c_int), ("cached", ctypes.c_int)]


class dgfs_profile_t(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("gain_launches", ctypes.c_int64),
                ("gain_timed", ctypes.c_int64), ("gain_ms", ctypes.c_double), ("nodes", ctypes.c_int64)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIGNATURES = {
    "dgfs_plan_desc_init": [ctypes.POINTER(dgfs_plan_desc)],
    "dgfs_plan_create": [ctypes.POINTER(dgfs_plan_desc), ctypes.POINTER(_P)],
    "dgfs_plan_destroy": [_P],
    "dgfs_plan_info": [_P, ctypes.POINTER(dgfs_plan_info_t)],
    "dgfs_collide": [_P, _P, _P, _I64, _P],
    "dgfs_collide2": [_P, _P, _P, _P, _I64, _P],
    "dgfs_collide_jvp": [_P, _P, _P, _P, _I64, _P],
    "dgfs_collide_vjp": [_P, _P, _P, _P, _I64, _P],
    "dgfs_collide_dgamma": [_P, _P, _P, _I64, _P],
    "dgfs_collide_ragged": [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_double), _I64, _P, _P, _P],
    "dgfs_ragged_create": [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                           ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double), _I64, ctypes.POINTER(_P)],
    "dgfs_ragged_collide": [_P, _P, _P, _P],
    "dgfs_ragged_destroy": [_P],
    "dgfs_collide_host": [_P, _P, _P, _I64, _P],
    "dgfs_collide_noalloc": [_P, _P, _P, _I64, _P],
    "dgfs_stream_status": [_P, _P],
    "dgfs_debug_inject": [_P, ctypes.c_int],
    "dgfs_device_fma_peaks": [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    "dgfs_device_mma_cycles": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)],
    "dgfs_plan_fingerprint": [_P, ctypes.POINTER(ctypes.c_uint64)],
    "dgfs_host_plan_fingerprint": [ctypes.POINTER(dgfs_plan_desc), ctypes.POINTER(ctypes.c_uint64)],
    "dgfs_host_pipeline_schedule": [ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                                    ctypes.POINTER(ctypes.c_int64)],
    "dgfs_plan_autotune": [_P, _P, _I64, _P, ctypes.POINTER(dgfs_tune_report)],
    "dgfs_plan_set_tuning": [_P, ctypes.c_int, _I64],
    "dgfs_profile_begin": [_P],
    "dgfs_profile_end": [_P, ctypes.POINTER(dgfs_profile_t)],
    "dgfs_last_error_message": [],
    "dgfs_host_quadrature": [ctypes.POINTER(dgfs_plan_desc), ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double)],
    "dgfs_host_translate_filter": [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_double)],
    "dgfs_ssprk": [_P, ctypes.c_int, _P, _I64, ctypes.c_double, ctypes.c_double, ctypes.c_int, _P],
    "dgfs_moments": [_P, _P, _P, _I64, _P],
    "dgfs_dg_create": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_double, _I64,
                       ctypes.POINTER(_P)],
    "dgfs_dg_info": [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "dgfs_dg_collide": [_P, _P, _P, _I64, _P],
    "dgfs_dg_destroy": [_P],
    "dgfs_host_dg_tensor": [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_double)],
    "dgfs_slab_create": [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                         ctypes.POINTER(_P)],
    "dgfs_slab_set_walls": [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    "dgfs_slab_rhs": [_P, _P, _P, _P],
    "dgfs_slab_ssprk": [_P, ctypes.c_int, _P, ctypes.c_double, ctypes.c_int, _P],
    "dgfs_slab_destroy": [_P],
    "dgfs_host_dg_stiffness": [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    "dgfs_host_vss_tables": [ctypes.POINTER(dgfs_plan_desc), ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double)],
    "dgfs_host_vss_factor": [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
}

_lib = None


def lib():
    """The loaded libdgfs.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libdgfs.so is not built (%s); run paper_1809_10186_gb300.build.build()"
                               % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_char_p if name == "dgfs_last_error_message" else ctypes.c_int
        _lib = L
    return _lib


class DGFSError(RuntimeError):
    def __init__(self, status, where):
        msg = lib().dgfs_last_error_message().decode()
        super().__init__("%s failed: %s (%s)" % (where, STATUS.get(status, status), msg))
        self.status = status


def check(status, where):
    if status != 0:
        raise DGFSError(status, where)


def make_desc(N=32, L=7.0, gamma=0.0, b=0.0, R=0.0, M=38, N_rho=0, svd_tol=0.0, svd_rank=0,
              precision="fp32", loss="paper", max_batch=0, sphere=None, alpha=0.0):
    d = dgfs_plan_desc()
    check(lib().dgfs_plan_desc_init(ctypes.byref(d)), "dgfs_plan_desc_init")
    d.N, d.L, d.gamma, d.b, d.R, d.M = int(N), float(L), float(gamma), float(b or 0.0), float(R or 0.0), int(M)
    d.N_rho, d.svd_tol, d.svd_rank = int(N_rho or 0), float(svd_tol), int(svd_rank)
    d.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    d.loss_mode = LOSS_MODES[loss] if isinstance(loss, str) else int(loss)
    d.max_batch = int(max_batch)
    d.alpha = float(alpha or 0.0)
    keep = None
    if sphere is not None:
        import numpy as np
        keep = np.ascontiguousarray(sphere, dtype=np.float64)
        d.M = 2 * keep.shape[0]
        d.sphere_xyzw = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return d, keep


def host_quadrature(**kw):
    """(c_r, w_r, sigma_xyzw, R, b) of the plan builder, without touching the GPU."""
    import numpy as np
    d, keep = make_desc(**kw)
    npairs = ctypes.c_int(0)
    R, b = ctypes.c_double(0), ctypes.c_double(0)
    check(lib().dgfs_host_quadrature(ctypes.byref(d), None, None, None, ctypes.byref(npairs),
                                     ctypes.byref(R), ctypes.byref(b)), "dgfs_host_quadrature")
    nr = d.N_rho if d.N_rho > 0 else d.N
    cr, wr = np.zeros(nr), np.zeros(nr)
    sig = np.zeros((npairs.value, 4))
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    check(lib().dgfs_host_quadrature(ctypes.byref(d), dp(cr), dp(wr), dp(sig), ctypes.byref(npairs),
                                     None, None), "dgfs_host_quadrature")
    return cr, wr, sig, R.value, b.value


def host_translate_filter(N, L, t):
    import numpy as np
    a = np.zeros(N)
    check(lib().dgfs_host_translate_filter(int(N), float(L), float(t),
                                           a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
          "dgfs_host_translate_filter")
    return a


def host_vss_factor(L, gamma, alpha, k_abs, mu, c_r, b=0.0):
    """The plan builder's F(k, c_r, sigma) of the VSS kernel at the given points (host, no GPU)."""
    import numpy as np
    k_abs, mu, c_r = np.broadcast_arrays(*(np.ascontiguousarray(x, dtype=np.float64) for x in (k_abs, mu, c_r)))
    k_abs, mu, c_r = (np.ascontiguousarray(x).ravel() for x in (k_abs, mu, c_r))
    out = np.zeros(len(k_abs))
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    check(lib().dgfs_host_vss_factor(float(L), float(gamma), float(b), float(alpha), len(out), dp(k_abs), dp(mu),
                                     dp(c_r), dp(out)), "dgfs_host_vss_factor")
    return out


def host_vss_tables(**kw):
    """(A [N_rho, n_pairs, N, N, N], GL [N, N, N]) of a VSS plan, built on the host, DFT index order."""
    import numpy as np
    _, _, sig, _, _ = host_quadrature(**kw)
    d, keep = make_desc(**kw)
    N, nr = d.N, (d.N_rho if d.N_rho > 0 else d.N)
    A = np.zeros((nr, sig.shape[0], N, N, N))
    GL = np.zeros((N, N, N))
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    check(lib().dgfs_host_vss_tables(ctypes.byref(d), dp(A), dp(GL)), "dgfs_host_vss_tables")
    return A, GL


def host_plan_fingerprint(**kw):
    """64-bit fingerprint of the plan a descriptor builds (dgfs_host_plan_fingerprint; no GPU)."""
    d, _keep = make_desc(**kw)
    out = ctypes.c_uint64(0)
    check(lib().dgfs_host_plan_fingerprint(ctypes.byref(d), ctypes.byref(out)), "dgfs_host_plan_fingerprint")
    return out.value


def host_pipeline_schedule(B, chunk):
    """Sub-batch sizes of the host-buffer pipeline for B nodes and a plan chunk (no GPU)."""
    n = ctypes.c_int64(0)
    check(lib().dgfs_host_pipeline_schedule(B, chunk, None, 0, ctypes.byref(n)), "dgfs_host_pipeline_schedule")
    buf = (ctypes.c_int64 * max(1, n.value))()
    check(lib().dgfs_host_pipeline_schedule(B, chunk, buf, n.value, ctypes.byref(n)), "dgfs_host_pipeline_schedule")
    return [buf[i] for i in range(n.value)]


def device_fma_peaks():
    """(FP32, FP64) FMA throughput of the current device in TFLOP/s, measured (dgfs_device_fma_peaks)."""
    a, b = ctypes.c_double(0), ctypes.c_double(0)
    check(lib().dgfs_device_fma_peaks(ctypes.byref(a), ctypes.byref(b)), "dgfs_device_fma_peaks")
    return a.value, b.value


def device_mma_cycles(n, a_from_tmem=False):
    """SM cycles per back-to-back tcgen05 MMA of M = 128, K = 16, N = n (dgfs_device_mma_cycles)."""
    c = ctypes.c_double(0)
    check(lib().dgfs_device_mma_cycles(int(n), 1 if a_from_tmem else 0, ctypes.byref(c)), "dgfs_device_mma_cycles")
    return c.value


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """Owns one dgfs_plan_t. Methods take CUDA tensors [B, N, N, N] and return new tensors."""

    def __init__(self, **kw):
        d, keep = make_desc(**kw)
        h = ctypes.c_void_p()
        check(lib().dgfs_plan_create(ctypes.byref(d), ctypes.byref(h)), "dgfs_plan_create")
        self.handle = h
        info = dgfs_plan_info_t()
        check(lib().dgfs_plan_info(h, ctypes.byref(info)), "dgfs_plan_info")
        self.info = {k: getattr(info, k) for k, _ in dgfs_plan_info_t._fields_}
        self.N = info.N
        self.precision = kw.get("precision", "fp32")

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == "fp64" else torch.float32

    def close(self):
        if getattr(self, "handle", None):
            lib().dgfs_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_field(self, t, name):
        import torch
        if not (t.is_cuda and t.dtype == self.dtype and t.is_contiguous()
                and t.dim() == 4 and tuple(t.shape[1:]) == (self.N,) * 3):
            raise ValueError("%s must be a contiguous CUDA %s tensor [B, %d, %d, %d]"
                             % (name, self.dtype, self.N, self.N, self.N))

    def _call(self, fn_name, fields, out=None, stream=None):
        import torch
        for i, t in enumerate(fields):
            self._check_field(t, "arg%d" % i)
        if out is None:
            out = torch.empty_like(fields[0])
        self._check_field(out, "out")
        ptrs = [ctypes.c_void_p(t.data_ptr()) for t in fields]
        fn = getattr(lib(), fn_name)
        check(fn(self.handle, *ptrs, ctypes.c_void_p(out.data_ptr()), ctypes.c_int64(fields[0].shape[0]),
                 _stream_ptr(stream)), fn_name)
        return out

    def collide(self, f, out=None, stream=None):
        return self._call("dgfs_collide", [f], out, stream)

    def collide_noalloc(self, f, out=None, stream=None):
        """Q(f, f) with scratch in the library's fixed device array (no device allocation)."""
        return self._call("dgfs_collide_noalloc", [f], out, stream)

    def collide2(self, f, g, out=None, stream=None):
        return self._call("dgfs_collide2", [f, g], out, stream)

    def collide_jvp(self, f, v, out=None, stream=None):
        return self._call("dgfs_collide_jvp", [f, v], out, stream)

    def collide_vjp(self, f, u, out=None, stream=None):
        return self._call("dgfs_collide_vjp", [f, u], out, stream)

    def collide_dgamma(self, f, out=None, stream=None):
        return self._call("dgfs_collide_dgamma", [f], out, stream)

    def collide_host(self, f_host, q_host, stream=None):
        """f_host, q_host: CPU tensors (pinned for overlap); copies are inside the call."""
        B = f_host.shape[0]
        check(lib().dgfs_collide_host(self.handle, ctypes.c_void_p(f_host.data_ptr()),
                                      ctypes.c_void_p(q_host.data_ptr()), ctypes.c_int64(B),
                                      _stream_ptr(stream)), "dgfs_collide_host")
        return q_host

    def autotune(self, f, stream=None):
        """Times the candidate configurations on f and keeps the fastest (dgfs_plan_autotune); returns
        the report as a dict."""
        self._check_field(f, "f")
        rep = dgfs_tune_report()
        check(lib().dgfs_plan_autotune(self.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_int64(f.shape[0]),
                                       _stream_ptr(stream), ctypes.byref(rep)), "dgfs_plan_autotune")
        return {k: getattr(rep, k) for k, _ in dgfs_tune_report._fields_}

    def set_tuning(self, rpc=0, chunk_nodes=0):
        check(lib().dgfs_plan_set_tuning(self.handle, int(rpc), ctypes.c_int64(chunk_nodes)), "dgfs_plan_set_tuning")

    def fingerprint(self):
        """64-bit fingerprint of the plan's tables (dgfs_plan_fingerprint)."""
        out = ctypes.c_uint64(0)
        check(lib().dgfs_plan_fingerprint(self.handle, ctypes.byref(out)), "dgfs_plan_fingerprint")
        return out.value

    def profile_begin(self):
        check(lib().dgfs_profile_begin(self.handle), "dgfs_profile_begin")

    def profile_end(self):
        out = dgfs_profile_t()
        check(lib().dgfs_profile_end(self.handle, ctypes.byref(out)), "dgfs_profile_end")
        return {k: getattr(out, k) for k, _ in dgfs_profile_t._fields_}

    def stream_status(self, stream=None):
        check(lib().dgfs_stream_status(self.handle, _stream_ptr(stream)), "dgfs_stream_status")

    def ssprk(self, f, dt, steps, order=2, scale=1.0, stream=None):
        """Advances df/dt = scale Q(f, f) in place by `steps` SSP-RK steps (dgfs_ssprk)."""
        check(lib().dgfs_ssprk(self.handle, int(order), ctypes.c_void_p(f.data_ptr()), ctypes.c_int64(f.shape[0]),
                               float(dt), float(scale), int(steps), _stream_ptr(stream)), "dgfs_ssprk")
        return f

    MOMENT_NAMES = ("n", "ux", "uy", "uz", "T", "Pxx", "Pyy", "Pzz", "Pxy", "Pxz", "Pyz", "qx", "qy", "qz", "H")

    def moments(self, f, stream=None):
        """[B, 15] float64 device tensor: n, u, T, P, q and H of every node (dgfs_moments)."""
        import torch
        out = torch.empty(f.shape[0], 15, dtype=torch.float64, device=f.device)
        check(lib().dgfs_moments(self.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_int64(f.shape[0]), _stream_ptr(stream)), "dgfs_moments")
        return out

    def debug_inject(self, mode=1):
        """Failure-detection test hook: mode 1 makes the next tensor-core launch lose one
        hand-off signal in its first CTA (see dgfs_debug_inject)."""
        check(lib().dgfs_debug_inject(self.handle, int(mode)), "dgfs_debug_inject")


def collide_ragged(plans, node_plan, node_offset, f_packed, node_gamma=None, node_b=None,
                   out=None, stream=None):
    """Q for a packed batch of nodes with mixed N (one plan per N). Host arrays for the layout."""
    import numpy as np
    import torch
    node_plan = np.ascontiguousarray(node_plan, dtype=np.int32)
    node_offset = np.ascontiguousarray(node_offset, dtype=np.int64)
    B = node_plan.shape[0]
    if out is None:
        out = torch.empty_like(f_packed)
    handles = (ctypes.c_void_p * len(plans))(*[p.handle for p in plans])
    gptr = bptr = None
    if node_gamma is not None:
        node_gamma = np.ascontiguousarray(node_gamma, dtype=np.float64)
        gptr = node_gamma.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if node_b is not None:
        node_b = np.ascontiguousarray(node_b, dtype=np.float64)
        bptr = node_b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    check(lib().dgfs_collide_ragged(handles, len(plans),
                                    node_plan.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                    node_offset.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                    gptr, bptr, ctypes.c_int64(B), ctypes.c_void_p(f_packed.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
          "dgfs_collide_ragged")
    return out


class RaggedSchedule:
    """A mixed-N node layout prepared once (dgfs_ragged_create): per-class node arrays live on the
    device, so collide() issues kernel launches only and can be captured in a CUDA graph."""

    def __init__(self, plans, node_plan, node_offset, node_gamma=None, node_b=None):
        import numpy as np
        node_plan = np.ascontiguousarray(node_plan, dtype=np.int32)
        node_offset = np.ascontiguousarray(node_offset, dtype=np.int64)
        self.plans = list(plans)   # the plans must outlive the schedule
        handles = (ctypes.c_void_p * len(plans))(*[p.handle for p in plans])
        gptr = bptr = None
        if node_gamma is not None:
            node_gamma = np.ascontiguousarray(node_gamma, dtype=np.float64)
            gptr = node_gamma.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if node_b is not None:
            node_b = np.ascontiguousarray(node_b, dtype=np.float64)
            bptr = node_b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        h = ctypes.c_void_p()
        check(lib().dgfs_ragged_create(handles, len(plans), node_plan.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                       node_offset.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), gptr, bptr,
                                       ctypes.c_int64(node_plan.shape[0]), ctypes.byref(h)),
              "dgfs_ragged_create")
        self.handle = h

    def collide(self, f_packed, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(f_packed)
        check(lib().dgfs_ragged_collide(self.handle, ctypes.c_void_p(f_packed.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
              "dgfs_ragged_collide")
        return out

    def close(self):
        if getattr(self, "handle", None):
            lib().dgfs_ragged_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def host_dg_tensor(K):
    """Gauss-Lobatto nodes, mass matrix and H[m][l1][l2] of the 1-D nodal DG basis (host only)."""
    import numpy as np
    nodes, M, H = np.zeros(K), np.zeros((K, K)), np.zeros((K, K, K))
    dp = ctypes.POINTER(ctypes.c_double)
    check(lib().dgfs_host_dg_tensor(int(K), nodes.ctypes.data_as(dp), M.ctypes.data_as(dp), H.ctypes.data_as(dp)),
          "dgfs_host_dg_tensor")
    return nodes, M, H


class DGElement:
    """The DG element collision term in the SVD variant (dgfs_dg_*): collide(F) maps the nodal
    distribution functions F [E, K, N, N, N] of E elements to C[e, m] = sum H[m, l1, l2] Q(F_l1, F_l2)."""

    def __init__(self, plan, H, svd_tol=0.0, max_elements=64):
        import numpy as np
        H = np.ascontiguousarray(H, dtype=np.float64)
        self.K = H.shape[0]
        self.plan = plan   # the plan must outlive this object
        h = ctypes.c_void_p()
        check(lib().dgfs_dg_create(plan.handle, self.K, H.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   float(svd_tol), ctypes.c_int64(max_elements), ctypes.byref(h)), "dgfs_dg_create")
        self.handle = h
        ranks = (ctypes.c_int * self.K)()
        total = ctypes.c_int()
        check(lib().dgfs_dg_info(h, ranks, ctypes.byref(total)), "dgfs_dg_info")
        self.ranks, self.total_rank = list(ranks), total.value

    def collide(self, F, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(F)
        check(lib().dgfs_dg_collide(self.handle, ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_int64(F.shape[0]), _stream_ptr(stream)), "dgfs_dg_collide")
        return out

    def close(self):
        if getattr(self, "handle", None):
            lib().dgfs_dg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def host_dg_stiffness(K):
    """(S, M^-1) of the K-node Gauss-Lobatto basis on [-1, 1] (S[m][l] = int phi_l phi_m')."""
    import numpy as np
    S, Mi = np.zeros((K, K)), np.zeros((K, K))
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    check(lib().dgfs_host_dg_stiffness(int(K), dp(S), dp(Mi)), "dgfs_host_dg_stiffness")
    return S, Mi


class Slab:
    """The 1-D DGFS solver (dgfs_slab_*): I elements of K nodes between two diffuse walls.
    F: CUDA tensor [I, K, N, N, N] of the plan's dtype. walls: (u_x, u_y, u_z, T_w), u_x = 0."""

    def __init__(self, plan, K, edges, Kn, wall_left, wall_right, svd_tol=0.0):
        import numpy as np
        edges = np.ascontiguousarray(edges, dtype=np.float64)
        self.K, self.I, self.plan = int(K), len(edges) - 1, plan   # the plan must outlive the slab
        wl, wr = (np.ascontiguousarray(w, dtype=np.float64) for w in (wall_left, wall_right))
        dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        h = ctypes.c_void_p()
        check(lib().dgfs_slab_create(plan.handle, self.K, self.I, dp(edges), float(Kn), dp(wl), dp(wr),
                                     float(svd_tol), ctypes.byref(h)), "dgfs_slab_create")
        self.handle = h

    def set_walls(self, wall_left, wall_right):
        import numpy as np
        wl, wr = (np.ascontiguousarray(w, dtype=np.float64) for w in (wall_left, wall_right))
        dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        check(lib().dgfs_slab_set_walls(self.handle, dp(wl), dp(wr)), "dgfs_slab_set_walls")

    def rhs(self, F, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(F)
        check(lib().dgfs_slab_rhs(self.handle, ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  _stream_ptr(stream)), "dgfs_slab_rhs")
        return out

    def ssprk(self, F, dt, steps, order=2, stream=None):
        check(lib().dgfs_slab_ssprk(self.handle, int(order), ctypes.c_void_p(F.data_ptr()), float(dt), int(steps),
                                    _stream_ptr(stream)), "dgfs_slab_ssprk")
        return F

    def close(self):
        if getattr(self, "handle", None):
            lib().dgfs_slab_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd_function():
    import torch

    class CollideFunction(torch.autograd.Function):
        """Q(f, f) of a plan, differentiable with respect to f and to the VHS exponent gamma.

        Reverse mode: the gradient of f is dgfs_collide_vjp(f, gQ); the gradient of gamma is the
        contraction sum_j gQ_j (dQ/dgamma)_j with dQ/dgamma from dgfs_collide_dgamma (b held fixed),
        per node for a gamma of shape [B], summed over the batch for a scalar gamma. Forward mode:
        dgfs_collide_jvp(f, v) + (dQ/dgamma) gamma_dot. The kernels recompute every translate;
        nothing but f is saved."""

        @staticmethod
        def forward(plan, f, gamma):
            return plan.collide(f.contiguous())

        @staticmethod
        def setup_context(ctx, inputs, output):
            plan, f, gamma = inputs
            ctx.plan = plan
            ctx.gamma_shape = None if gamma is None else tuple(gamma.shape)
            ctx.save_for_backward(f)
            ctx.f_fwd = f

        @staticmethod
        def backward(ctx, gQ):
            (f,) = ctx.saved_tensors
            f, gQ = f.contiguous(), gQ.contiguous()
            gf = ctx.plan.collide_vjp(f, gQ) if ctx.needs_input_grad[1] else None
            gg = None
            if ctx.gamma_shape is not None and ctx.needs_input_grad[2]:
                per_node = (gQ * ctx.plan.collide_dgamma(f)).sum(dim=(1, 2, 3))
                gg = per_node.sum() if len(ctx.gamma_shape) == 0 else per_node.reshape(ctx.gamma_shape)
            return None, gf, gg

        @staticmethod
        def jvp(ctx, _plan_t, v, gamma_t):
            f = ctx.f_fwd.contiguous()
            out = ctx.plan.collide_jvp(f, v.contiguous()) if v is not None else None
            if gamma_t is not None:
                scale = gamma_t.reshape(-1, 1, 1, 1) if gamma_t.dim() else gamma_t
                dg = ctx.plan.collide_dgamma(f) * scale
                out = dg if out is None else out + dg
            return out if out is not None else torch.zeros_like(f)

    return CollideFunction


_CF = None


def collide(plan, f, gamma=None):
    """Differentiable Q(f, f) (torch.autograd reverse and forward mode).

    gamma: None, or a tensor (scalar, or [B] for one value per node) holding the plan's VHS
    exponent; gradients flow to it through dQ/dgamma at fixed b. The plan's tables are built for
    its gamma, so the values must equal it: to move gamma (e.g. in a fit), build a plan at the new
    value (the host plan builder takes milliseconds) and call again."""
    global _CF
    if _CF is None:
        _CF = _autograd_function()
    if gamma is not None:
        import torch
        if not torch.is_tensor(gamma) or gamma.dim() > 1 or (gamma.dim() == 1 and gamma.shape[0] != f.shape[0]):
            raise ValueError("gamma must be a scalar tensor or a tensor of shape [B]")
        if torch.any(torch.abs(gamma.detach().double() - plan.info["gamma"]) > 1e-12 * max(1.0, abs(plan.info["gamma"]))):
            raise ValueError("gamma must equal the plan's gamma (%r); build a plan at the new value"
                             % plan.info["gamma"])
    return _CF.apply(plan, f, gamma)
