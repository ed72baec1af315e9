"""Python binding of libonmf: online and batch Itakura-Saito NMF on GB300.

Thin ctypes marshalling over the C ABI declared in ``include/onmf.h``; the
functions keep the C names. Every step of the computation runs in the CUDA
kernels of ``libonmf.so``; there is no Python or CPU fallback, and loading
fails loudly when the library cannot be built or loaded.

Arrays follow the library's memory order: a frame-major spectrogram V is a
(n, F) array (row j = frame j = column j of the F x n matrix), W is (K, F),
H is (n, K). Arguments may be torch tensors (CUDA or CPU) or numpy arrays;
the library detects whether a pointer is host or device memory.
"""
import ctypes
import os

import numpy as np

from ._build import LIB, build as _build_lib

__all__ = [
    "OnmfError", "onmf_config", "ONMF_FP32", "ONMF_MIXED", "lib", "build",
    "onmf_config_default", "onmf_init", "onmf_push_frames", "onmf_flush",
    "onmf_synchronize", "onmf_get_W", "onmf_get_stats", "onmf_set_state",
    "onmf_project", "nmf_batch_step", "nmf_batch_init_H", "onmf_destroy",
    "onmf_status_string", "onmf_kernel_launches", "onmf_abi_version",
    "onmf_project_static", "onmf_push_frames_warm", "onmf_autotune", "OnlineISNMF", "EXPORTED",
    "BatchPlan",
]

ONMF_FP32 = 0
ONMF_MIXED = 1
# h-solve kernels of the mixed path (onmf_config.hsolve)
ONMF_HSOLVE_AUTO, ONMF_HSOLVE_MMA, ONMF_HSOLVE_TC, ONMF_HSOLVE_CLUSTER = 0, 1, 2, 3
HSOLVE_NAMES = {0: "auto", 1: "mma", 2: "tc", 3: "cluster"}
ONMF_SERVE_GRAPH, ONMF_SERVE_DIRECT = 0, 1
ONMF_ACC_FP64, ONMF_ACC_FP32, ONMF_ACC_FP32_COMP = 0, 1, 2
ONMF_DEVERR_INPUT, ONMF_DEVERR_NUMERIC, ONMF_DEVERR_TIMEOUT, ONMF_DEVERR_CONFIG = 1, 2, 4, 8
ACC_NAMES = {0: "fp64", 1: "fp32", 2: "fp32_compensated"}
ONMF_ETIMEOUT = 6

# Every symbol include/onmf.h declares.
EXPORTED = [
    "onmf_config_default", "onmf_init", "onmf_push_frames", "onmf_flush",
    "onmf_synchronize", "onmf_get_W", "onmf_get_stats", "onmf_set_state",
    "onmf_project", "nmf_batch_step", "nmf_batch_init_H", "onmf_destroy",
    "onmf_status_string", "onmf_last_error_message", "onmf_kernel_launches",
    "onmf_abi_version", "onmf_project_static",
    "onmf_server_create", "onmf_server_open_stream", "onmf_server_submit",
    "onmf_server_poll", "onmf_server_get_W", "onmf_server_close_stream",
    "onmf_server_get_stats", "onmf_server_destroy", "onmf_selftest_wait",
    "onmf_push_frames_warm", "onmf_autotune", "onmf_server_submit_many",
    "nmf_batch_plan_create", "nmf_batch_plan_step", "nmf_batch_plan_destroy",
]


class onmf_config(ctypes.Structure):
    _fields_ = [
        ("F", ctypes.c_int32), ("K", ctypes.c_int32),
        ("beta", ctypes.c_int32), ("n_inner", ctypes.c_int32),
        ("eps", ctypes.c_double), ("r", ctypes.c_double),
        ("n_ref", ctypes.c_int64), ("h_exponent", ctypes.c_double),
        ("normalize", ctypes.c_int32), ("rho_on_new", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("hsolve", ctypes.c_int32),
        ("accumulate", ctypes.c_int32), ("stats_ranges", ctypes.c_int32),
        ("h_penalty", ctypes.c_double), ("h_penalty_a", ctypes.c_double),
        ("w_penalty", ctypes.c_double),
    ]


class onmf_server_config(ctypes.Structure):
    _fields_ = [
        ("F", ctypes.c_int32), ("max_chunk", ctypes.c_int32),
        ("max_batch", ctypes.c_int32), ("slots", ctypes.c_int32),
        ("budget_bytes", ctypes.c_int64), ("precision", ctypes.c_int32),
        ("launch", ctypes.c_int32),
    ]


class onmf_completion(ctypes.Structure):
    _fields_ = [
        ("stream_id", ctypes.c_int64), ("tag", ctypes.c_int64),
        ("frames", ctypes.c_int64), ("loss", ctypes.c_double),
        ("t_submit", ctypes.c_double), ("t_done", ctypes.c_double),
        ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class onmf_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "launches", "chunks", "frames", "batches_overlapped",
        "streams_admitted", "streams_pending", "bytes_in_use", "host_batch_ns",
        "device_ns")]


class OnmfError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        msg = onmf_status_string(status)
        detail = lib().onmf_last_error_message().decode(errors="replace")
        super().__init__("%s%s%s" % (where + ": " if where else "", msg,
                                     " (" + detail + ")" if detail else ""))


_LIB = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_d = ctypes.c_double


def build(force=False):
    """Compile libonmf.so for sm_103a (nvcc) and return its path."""
    return _build_lib(force=force)


def lib():
    """Load libonmf.so, building it first if it is missing or stale. With
    ONMF_LIB_VARIANT=phase in the environment, the phase-timing build
    (identical kernels plus clock64 stamps at the phase boundaries)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    variant = os.environ.get("ONMF_LIB_VARIANT") or None
    path = _build_lib(variant=variant)
    L = ctypes.CDLL(path)
    L.onmf_config_default.argtypes = [ctypes.POINTER(onmf_config), _i32, _i32]
    L.onmf_config_default.restype = None
    L.onmf_init.argtypes = [ctypes.POINTER(onmf_config), _vp, _i32, _vp,
                            ctypes.POINTER(_vp)]
    L.onmf_push_frames.argtypes = [_vp, _vp, _i64, _i64, _vp, _i64]
    L.onmf_push_frames_warm.argtypes = [_vp, _vp, _i64, _i64, _vp, _vp, _i64]
    L.onmf_autotune.argtypes = [ctypes.POINTER(onmf_config), _vp, ctypes.c_char_p,
                                ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                ctypes.POINTER(_d * 4), ctypes.POINTER(_d * 5),
                                ctypes.POINTER(_i32)]
    L.onmf_flush.argtypes = [_vp]
    L.onmf_synchronize.argtypes = [_vp]
    L.onmf_get_W.argtypes = [_vp, _vp, _i32]
    L.onmf_get_stats.argtypes = [_vp, _vp, _vp, ctypes.POINTER(_i64),
                                 ctypes.POINTER(_d)]
    L.onmf_set_state.argtypes = [_vp, _vp, _vp, _vp, _i64, _d]
    L.onmf_project.argtypes = [_vp, _vp, _i64, _i64, _vp, _i64, _i32,
                               ctypes.POINTER(_d)]
    L.nmf_batch_step.argtypes = [_vp, _i64, _vp, _vp, _i32, _i32, _i64, _d, _d,
                                 _i32, _i32, _i32, _vp, _vp]
    L.nmf_batch_init_H.argtypes = [_vp, _i64, _vp, _vp, _i32, _i32, _i64, _d,
                                   _vp]
    L.nmf_batch_plan_create.argtypes = [_i32, _i32, _i64, _i32, ctypes.POINTER(_vp)]
    L.nmf_batch_plan_step.argtypes = [_vp, _vp, _i64, _vp, _vp, _i64, _d, _d, _i32,
                                      _i32, _vp, _vp]
    L.nmf_batch_plan_destroy.argtypes = [_vp]
    L.nmf_batch_plan_destroy.restype = None
    L.onmf_project_static.argtypes = [_vp, _i32, _i32, _vp, _i64, _i64, _vp,
                                      _i64, _d, _d, _i32, _i32, _vp, _vp, _vp]
    L.onmf_destroy.argtypes = [_vp]
    L.onmf_destroy.restype = None
    L.onmf_server_create.argtypes = [ctypes.POINTER(onmf_server_config),
                                     ctypes.POINTER(_vp)]
    L.onmf_server_open_stream.argtypes = [_vp, ctypes.POINTER(onmf_config), _vp,
                                          ctypes.POINTER(_i64)]
    L.onmf_server_submit.argtypes = [_vp, _i64, _vp, _i64, _i64, _vp, _i64]
    L.onmf_server_submit_many.argtypes = [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp,
                                          ctypes.POINTER(_i32)]
    L.onmf_server_poll.argtypes = [_vp, ctypes.POINTER(onmf_completion), _i32,
                                   ctypes.POINTER(_i32), _i32]
    L.onmf_server_get_W.argtypes = [_vp, _i64, _vp]
    L.onmf_server_close_stream.argtypes = [_vp, _i64]
    L.onmf_server_get_stats.argtypes = [_vp, ctypes.POINTER(onmf_server_stats)]
    L.onmf_server_destroy.argtypes = [_vp]
    L.onmf_server_destroy.restype = None
    L.onmf_status_string.argtypes = [ctypes.c_int]
    L.onmf_status_string.restype = ctypes.c_char_p
    L.onmf_last_error_message.restype = ctypes.c_char_p
    L.onmf_kernel_launches.restype = _i64
    L.onmf_abi_version.restype = _i32
    L.onmf_selftest_wait.argtypes = [_i32, _vp, ctypes.POINTER(_i64)]
    for name in ("onmf_init", "onmf_push_frames", "onmf_flush",
                 "onmf_synchronize", "onmf_get_W", "onmf_get_stats",
                 "onmf_set_state", "onmf_project", "nmf_batch_step",
                 "nmf_batch_init_H", "onmf_project_static", "onmf_server_create",
                 "onmf_server_open_stream", "onmf_server_submit", "onmf_server_poll",
                 "onmf_server_get_W", "onmf_server_close_stream",
                 "onmf_server_get_stats", "onmf_selftest_wait", "onmf_push_frames_warm",
                 "onmf_autotune", "onmf_server_submit_many", "nmf_batch_plan_create",
                 "nmf_batch_plan_step"):
        getattr(L, name).restype = ctypes.c_int
    _LIB = L
    return L


def _check(st, where):
    if st != 0:
        raise OnmfError(st, where)


# ------------------------------------------------------------ marshalling


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr_ld(x, cols):
    """(pointer, leading dimension) of a 2-D row-major array with `cols`
    columns whose rows may be strided (row stride = leading dimension)."""
    if x is None:
        return None, 0
    if _is_torch(x):
        import torch
        assert x.dtype in (torch.float32, torch.float64), x.dtype
        assert x.dim() == 2 and x.shape[1] == cols and x.stride(1) == 1, \
            "expected (n, %d) with unit column stride" % cols
        return x.data_ptr(), max(x.stride(0), cols)
    assert isinstance(x, np.ndarray) and x.ndim == 2 and x.shape[1] == cols
    assert x.strides[1] == x.itemsize, "rows must be contiguous"
    return x.ctypes.data, max(x.strides[0] // x.itemsize, cols)


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return 0
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# -------------------------------------------------------------- C names


def onmf_status_string(st):
    return lib().onmf_status_string(int(st)).decode()


def onmf_kernel_launches():
    return int(lib().onmf_kernel_launches())


def onmf_abi_version():
    return int(lib().onmf_abi_version())


def onmf_selftest_wait(which, stream=None):
    """Run bounded wait `which` (0 grid barrier, 1 mbarrier, 2 mbarrier with
    tensor memory held) on a condition that never holds. Returns
    (status, elapsed device ns); the expected status is ONMF_ETIMEOUT."""
    el = _i64(0)
    st = lib().onmf_selftest_wait(int(which), _stream_handle(stream), ctypes.byref(el))
    return int(st), int(el.value)


def onmf_config_default(F, K, **kw):
    c = onmf_config()
    lib().onmf_config_default(ctypes.byref(c), int(F), int(K))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def onmf_init(cfg, W0, stream=None):
    """Create an online state from W0 (K, F) float32 (host or device)."""
    if _is_torch(W0):
        W0 = W0.contiguous()
        assert W0.dtype.is_floating_point and W0.element_size() == 4
        p = W0.data_ptr()
        keep = W0
    else:
        keep = np.ascontiguousarray(W0, dtype=np.float32)
        p = keep.ctypes.data
    assert tuple(keep.shape) == (cfg.K, cfg.F), "W0 must be (K, F)"
    h = _vp()
    _check(lib().onmf_init(ctypes.byref(cfg), p, 0, _stream_handle(stream),
                           ctypes.byref(h)), "onmf_init")
    return h


def onmf_push_frames(state, V, H_out=None, n=None):
    """Push frames V (n, F) float32; optional H_out (n, K) receives h."""
    K = H_out.shape[1] if H_out is not None else 1
    pv, ldv = _ptr_ld(V, V.shape[1])
    ph, ldh = _ptr_ld(H_out, K) if H_out is not None else (None, 1)
    n = V.shape[0] if n is None else n
    _check(lib().onmf_push_frames(state, pv, ldv, n, ph, ldh), "onmf_push_frames")


def onmf_push_frames_warm(state, V, H, order=None):
    """Warm-restart pass over device frames V (N, F): frames V[order[i]] in
    order (all rows if order is None), each h-solve starting from H[order[i]]
    (device (N, K), updated in place). order: int64 device tensor or None."""
    pv, ldv = _ptr_ld(V, V.shape[1])
    ph, ldh = _ptr_ld(H, H.shape[1])
    if order is not None:
        import torch
        assert order.dtype == torch.int64 and order.is_cuda and order.is_contiguous()
        n, po = order.numel(), order.data_ptr()
    else:
        n, po = V.shape[0], None
    _check(lib().onmf_push_frames_warm(state, pv, ldv, n, po, ph, ldh), "onmf_push_frames_warm")


STATS_RANGE_CANDIDATES = (0, 2, 4, 8, 16)


def onmf_autotune(cfg, cache_path=None, stream=None):
    """Time every schedule of the mixed online step the shape of cfg allows
    (h-solve kernel; with the mma kernel, the statistics' frame ranges).
    Returns (hsolve, stats_ranges, {kernel name: best us per minibatch},
    {stats_ranges: us per minibatch of the mma kernel}, from_cache)."""
    h = _i32(0)
    sr = _i32(0)
    us = (_d * 4)()
    rus = (_d * 5)()
    fc = _i32(0)
    _check(lib().onmf_autotune(ctypes.byref(cfg), _stream_handle(stream),
                               cache_path.encode() if cache_path else None,
                               ctypes.byref(h), ctypes.byref(sr), ctypes.byref(us),
                               ctypes.byref(rus), ctypes.byref(fc)),
           "onmf_autotune")
    times = {HSOLVE_NAMES[i]: us[i] for i in (1, 2, 3) if us[i] >= 0}
    ranges = {STATS_RANGE_CANDIDATES[i]: rus[i] for i in range(5) if rus[i] >= 0}
    return int(h.value), int(sr.value), times, ranges, bool(fc.value)


def onmf_flush(state):
    _check(lib().onmf_flush(state), "onmf_flush")


def onmf_synchronize(state):
    _check(lib().onmf_synchronize(state), "onmf_synchronize")


def onmf_get_W(state, out):
    """Copy W into `out` ((K, F) float32 tensor or array, host or device)."""
    p = out.data_ptr() if _is_torch(out) else out.ctypes.data
    _check(lib().onmf_get_W(state, p, 0), "onmf_get_W")
    return out


def onmf_get_stats(state, A=None, B=None):
    """Fill A, B ((K, F) float64 host arrays, optional); return (t, loss_sum)."""
    t = _i64(0)
    ls = _d(0.0)
    pa = A.ctypes.data if A is not None else None
    pb = B.ctypes.data if B is not None else None
    _check(lib().onmf_get_stats(state, pa, pb, ctypes.byref(t), ctypes.byref(ls)),
           "onmf_get_stats")
    return t.value, ls.value


def onmf_set_state(state, W, A, B, t, loss_sum):
    W = np.ascontiguousarray(W, dtype=np.float32)
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    _check(lib().onmf_set_state(state, W.ctypes.data, A.ctypes.data,
                                B.ctypes.data, int(t), float(loss_sum)),
           "onmf_set_state")


def onmf_project(state, V, H_out, n_inner=-1, want_obj=False):
    """h-solve of V (n, F) with W fixed into H_out (n, K); returns the d_IS
    sum when want_obj (synchronizing), else None."""
    pv, ldv = _ptr_ld(V, V.shape[1])
    ph, ldh = _ptr_ld(H_out, H_out.shape[1])
    obj = _d(0.0)
    _check(lib().onmf_project(state, pv, ldv, V.shape[0], ph, ldh, int(n_inner),
                              ctypes.byref(obj) if want_obj else None),
           "onmf_project")
    return obj.value if want_obj else None


def nmf_batch_init_H(V, W, H, eps=1e-12, stream=None):
    """Fresh-restart start point for every column of H (device tensors)."""
    pv, ldv = _ptr_ld(V, V.shape[1])
    K, F = W.shape
    _check(lib().nmf_batch_init_H(pv, ldv, W.data_ptr(), H.data_ptr(), F, K,
                                  V.shape[0], eps, _stream_handle(stream)),
           "nmf_batch_init_H")


def nmf_batch_step(V, W, H, eps=1e-12, h_exponent=0.5, n_iter=1, normalize=1,
                   precision=ONMF_FP32, want_obj=True, stream=None):
    """Batch IS-NMF cycles on device tensors V (N, F), W (K, F), H (N, K),
    updated in place. Returns the objective after each cycle (or None)."""
    pv, ldv = _ptr_ld(V, V.shape[1])
    K, F = W.shape
    N = V.shape[0]
    obj = (ctypes.c_double * max(1, n_iter))() if want_obj else None
    _check(lib().nmf_batch_step(pv, ldv, W.data_ptr(), H.data_ptr(), F, K, N, eps,
                                h_exponent, n_iter, normalize, precision,
                                obj, _stream_handle(stream)),
           "nmf_batch_step")
    return np.array(obj[:n_iter]) if want_obj else None


class BatchPlan:
    """Owner of an nmf_batch_plan: batch cycles of one shape (F, K, at most
    N_max frames, precision) with the scratch allocated once."""

    def __init__(self, F, K, N_max, precision=ONMF_FP32):
        self.F, self.K, self.N_max, self.precision = F, K, N_max, precision
        h = _vp()
        _check(lib().nmf_batch_plan_create(F, K, N_max, precision, ctypes.byref(h)),
               "nmf_batch_plan_create")
        self._h = h

    def step(self, V, W, H, eps=1e-12, h_exponent=0.5, n_iter=1, normalize=1,
             want_obj=True, stream=None):
        """nmf_batch_step on device tensors V (N, F), W (K, F), H (N, K)."""
        pv, ldv = _ptr_ld(V, V.shape[1])
        obj = (ctypes.c_double * max(1, n_iter))() if want_obj else None
        _check(lib().nmf_batch_plan_step(self._h, pv, ldv, W.data_ptr(), H.data_ptr(),
                                         V.shape[0], eps, h_exponent, n_iter, normalize,
                                         obj, _stream_handle(stream)),
               "nmf_batch_plan_step")
        return np.array(obj[:n_iter]) if want_obj else None

    def close(self):
        if self._h:
            lib().nmf_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def onmf_project_static(W, V, H_out=None, obj_sum=None, eps=1e-12,
                        h_exponent=0.5, n_inner=10, precision=ONMF_FP32,
                        err_out=None, stream=None):
    """Allocation-free projection: device tensors W (K, F), V (n, F), H_out
    (n, K) or None, obj_sum a 1-element float64 device tensor or None,
    err_out a 1-element int32 device tensor (receives the ONMF_DEVERR_* bits
    the kernels raise) or None."""
    K, F = W.shape
    pv, ldv = _ptr_ld(V, F)
    ph, ldh = _ptr_ld(H_out, K) if H_out is not None else (None, K)
    po = obj_sum.data_ptr() if obj_sum is not None else None
    pe = err_out.data_ptr() if err_out is not None else None
    _check(lib().onmf_project_static(W.data_ptr(), F, K, pv, ldv, V.shape[0], ph,
                                     ldh, eps, h_exponent, n_inner, precision,
                                     po, pe, _stream_handle(stream)),
           "onmf_project_static")


def onmf_destroy(state):
    if state:
        lib().onmf_destroy(state)


class OnlineISNMF:
    """Convenience owner of one online state (same calls, fewer arguments)."""

    def __init__(self, F, K, W0, stream=None, **cfg):
        self.cfg = onmf_config_default(F, K, **cfg)
        self.F, self.K = F, K
        self.state = onmf_init(self.cfg, W0, stream)

    def push(self, V, H_out=None):
        onmf_push_frames(self.state, V, H_out)

    def push_warm(self, V, H, order=None):
        onmf_push_frames_warm(self.state, V, H, order)

    def flush(self):
        onmf_flush(self.state)

    def sync(self):
        onmf_synchronize(self.state)

    def W(self):
        out = np.empty((self.K, self.F), dtype=np.float32)
        return onmf_get_W(self.state, out)

    def stats(self):
        A = np.empty((self.K, self.F))
        B = np.empty((self.K, self.F))
        t, ls = onmf_get_stats(self.state, A, B)
        return A, B, t, ls

    def set_state(self, W, A, B, t, loss_sum):
        onmf_set_state(self.state, W, A, B, t, loss_sum)

    def project(self, V, H_out, n_inner=-1, want_obj=False):
        return onmf_project(self.state, V, H_out, n_inner, want_obj)

    def close(self):
        if self.state:
            onmf_destroy(self.state)
            self.state = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- serving


def onmf_server_create(F, max_chunk=512, max_batch=256, slots=2,
                       budget_bytes=1 << 30, precision=ONMF_MIXED, launch=0):
    """launch: ONMF_SERVE_GRAPH (0, a captured CUDA graph per batch) or
    ONMF_SERVE_DIRECT (1, the phase kernels one by one)."""
    c = onmf_server_config(F, max_chunk, max_batch, slots, budget_bytes,
                           precision, launch)
    h = _vp()
    _check(lib().onmf_server_create(ctypes.byref(c), ctypes.byref(h)),
           "onmf_server_create")
    return h


def onmf_server_open_stream(srv, cfg, W0):
    W0 = np.ascontiguousarray(W0, dtype=np.float32)
    sid = _i64(0)
    _check(lib().onmf_server_open_stream(srv, ctypes.byref(cfg), W0.ctypes.data,
                                         ctypes.byref(sid)),
           "onmf_server_open_stream")
    return sid.value


def onmf_server_submit(srv, sid, V, tag=0, H_out=None):
    """Queue frames V (n, F) float32 host array; H_out (n, K) host array or None."""
    V = np.ascontiguousarray(V, dtype=np.float32)
    ph = H_out.ctypes.data if H_out is not None else None
    _check(lib().onmf_server_submit(srv, sid, V.ctypes.data, V.shape[1], V.shape[0],
                                    ph, int(tag)), "onmf_server_submit")


def onmf_server_submit_many(srv, sids, Vs, tags, H_outs=None):
    """Queue chunks Vs[i] ((n_i, F) float32 host arrays) for streams sids[i]
    in one call; H_outs: None or a list of (n_i, K) host arrays or None.
    Returns how many were queued (all, or raises at the first refused)."""
    m = len(Vs)
    Vs = [np.ascontiguousarray(v, dtype=np.float32) for v in Vs]
    pv = (ctypes.c_void_p * m)(*[v.ctypes.data for v in Vs])
    ld = (_i64 * m)(*[v.shape[1] for v in Vs])
    nn = (_i64 * m)(*[v.shape[0] for v in Vs])
    ids = (_i64 * m)(*[int(x) for x in sids])
    tg = (_i64 * m)(*[int(x) for x in tags])
    ph = None
    if H_outs is not None:
        ph = (ctypes.c_void_p * m)(*[h.ctypes.data if h is not None else None for h in H_outs])
    q = _i32(0)
    _check(lib().onmf_server_submit_many(srv, m, ids, pv, ld, nn, ph, tg, ctypes.byref(q)),
           "onmf_server_submit_many")
    return int(q.value)


def onmf_server_poll(srv, max_n=1024, wait_ms=0):
    buf = (onmf_completion * max_n)()
    n = _i32(0)
    _check(lib().onmf_server_poll(srv, buf, max_n, ctypes.byref(n), wait_ms),
           "onmf_server_poll")
    return [buf[i] for i in range(n.value)]


def onmf_server_get_W(srv, sid, K, F):
    W = np.empty((K, F), dtype=np.float32)
    _check(lib().onmf_server_get_W(srv, sid, W.ctypes.data), "onmf_server_get_W")
    return W


def onmf_server_close_stream(srv, sid):
    _check(lib().onmf_server_close_stream(srv, sid), "onmf_server_close_stream")


def onmf_server_get_stats(srv):
    st = onmf_server_stats()
    _check(lib().onmf_server_get_stats(srv, ctypes.byref(st)), "onmf_server_get_stats")
    return {n: getattr(st, n) for n, _ in onmf_server_stats._fields_}


def onmf_server_destroy(srv):
    if srv:
        lib().onmf_server_destroy(srv)
