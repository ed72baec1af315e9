"""FP64 CPU oracle for online and batch IS-NMF (arXiv:1106.4198).

TEST INFRASTRUCTURE ONLY: the plain, slow reference the CUDA path is checked
against. Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it. It shares no code with the CUDA library.

All arrays are numpy, column-major in the paper's sense: V is F x N with one
frame per column, W is F x K, H is K x N. Here they are passed as numpy
arrays of shape (N, F) for V (row n = frame n, contiguous), (K, F) for W
(row k = column k of W) and (N, K) for H, which is the same memory as the
column-major F x N / F x K / K x N matrices.
"""
import ctypes
import numpy as np

from .build import build_oracle

_LIB = None
_d = ctypes.c_double
_i = ctypes.c_int
_l = ctypes.c_int64
_p = ctypes.c_void_p


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build_oracle())
        lib.or_dis.restype = _d
        lib.or_dis.argtypes = [_p, _p, _l]
        lib.or_objective.restype = _d
        lib.or_objective.argtypes = [_i, _i, _l, _p, _l, _p, _p, _d]
        lib.or_hsolve.restype = None
        lib.or_hsolve.argtypes = [_i, _i, _p, _p, _d, _d, _i, _p, _p, _p]
        lib.or_hsolve_pen.restype = None
        lib.or_hsolve_pen.argtypes = [_i, _i, _p, _p, _d, _d, _i, _d, _d, _p, _p, _p]
        lib.or_stats_step.restype = None
        lib.or_stats_step.argtypes = [_i, _i, _l, _p, _l, _p, _d, _d, _i, _i,
                                      _p, _p, _p, _p]
        lib.or_stats_step_pen.restype = None
        lib.or_stats_step_pen.argtypes = [_i, _i, _l, _p, _l, _p, _d, _d, _i, _i, _d,
                                          _p, _p, _p, _p]
        lib.or_rho.restype = _d
        lib.or_rho.argtypes = [_d, _l, _l]
        lib.or_online_minibatch.restype = None
        lib.or_online_pass.restype = _l
        lib.or_online_pass.argtypes = [_i, _i, _l, _p, _l, _i, _i, _d, _d, _d,
                                       _l, _i, _i, _i, _d, _d, _d, _p, _p, _p, _p, _p,
                                       _p, _p]
        lib.or_project.restype = None
        lib.or_project.argtypes = [_i, _i, _l, _p, _l, _p, _d, _d, _i, _d, _d, _p, _p]
        lib.or_batch_h0.restype = None
        lib.or_batch_h0.argtypes = [_i, _i, _l, _p, _l, _p, _d, _p]
        lib.or_batch.restype = None
        lib.or_batch.argtypes = [_i, _i, _l, _p, _l, _p, _p, _d, _d, _i, _i,
                                 _p, _i]
        lib.or_set_threads.restype = None
        lib.or_set_threads.argtypes = [_i]
        lib.or_get_threads.restype = _i
        lib.or_have_openmp.restype = _i
        _LIB = lib
    return _LIB


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def set_threads(n):
    _lib().or_set_threads(int(n))


def get_threads():
    return _lib().or_get_threads()


def have_openmp():
    return bool(_lib().or_have_openmp())


def dis(y, x):
    """d_IS(y, x) summed over all entries (Section 2.1)."""
    y = _f64(y).ravel()
    x = _f64(x).ravel()
    assert y.shape == x.shape
    return _lib().or_dis(_ptr(y), _ptr(x), y.size)


def objective(V, W, H, eps):
    """(1/N) sum_n d_IS(eps + v_n, eps + W h_n); V (N,F), W (K,F), H (N,K)."""
    V = _f32(V)
    W = _f64(W)
    H = _f64(H)
    N, F = V.shape
    K = W.shape[0]
    return _lib().or_objective(F, K, N, _ptr(V), F, _ptr(W), _ptr(H), eps)


def hsolve(W, v, eps=1e-12, gamma=0.5, n_in=10, h_init=None, trace=False,
           h_penalty=0.0, h_penalty_a=1.0):
    """h-solve of one frame. W (K,F), v (F,). Returns h (K,) [, trace].
    h_penalty, h_penalty_a: lambda and a of the penalty lambda*log(a + sum h)
    (Section 2.2, "Extensions"); the trace then includes it."""
    W = _f64(W)
    v = _f32(v).ravel()
    K, F = W.shape
    h = np.zeros(K)
    hi = _f64(h_init) if h_init is not None else None
    tr = np.zeros(n_in + 1) if trace else None
    if h_penalty == 0.0:
        _lib().or_hsolve(F, K, _ptr(W), _ptr(v), eps, gamma, n_in, _ptr(hi),
                         _ptr(h), _ptr(tr))
    else:
        _lib().or_hsolve_pen(F, K, _ptr(W), _ptr(v), eps, gamma, n_in, h_penalty,
                             h_penalty_a, _ptr(hi), _ptr(h), _ptr(tr))
    return (h, tr) if trace else h


def stats_step(V, W, A, B, H, eps=1e-12, rho=1.0, normalize=True,
               rho_on_new=False, w_penalty=0.0):
    """Dictionary step given H. V (n,F); W, A, B (K,F); H (n,K); w_penalty:
    mu of the dictionary penalty mu*sum W. Returns (W, A, B, loss) as new
    arrays."""
    V = _f32(V)
    W = _f64(W).copy()
    A = _f64(A).copy()
    B = _f64(B).copy()
    H = _f64(H)
    n, F = V.shape
    K = W.shape[0]
    loss = ctypes.c_double(0.0)
    _lib().or_stats_step_pen(F, K, n, _ptr(V), F, _ptr(H), eps, rho, int(normalize),
                             int(rho_on_new), w_penalty, _ptr(W), _ptr(A), _ptr(B),
                             ctypes.byref(loss))
    return W, A, B, loss.value


def rho(r, nb, n_ref):
    return _lib().or_rho(r, nb, n_ref)


def online_pass(V, W, A=None, B=None, beta=50, n_in=5, eps=1e-12, gamma=0.5,
                r=1.0, n_ref=0, normalize=True, rho_on_new=False, flush=True,
                want_H=True, loss_sum=0.0, H_init=None, h_penalty=0.0,
                h_penalty_a=1.0, w_penalty=0.0):
    """One in-order pass of Algorithm 1. V (N,F), W (K,F) [A, B (K,F)];
    H_init (N,K): warm-restart start points of the frames' h-solves (None:
    fresh restarts); h_penalty, h_penalty_a, w_penalty: the penalties of
    Section 2.2 ("Extensions"). Returns dict(W, A, B, H (N,K) or None,
    loss_sum, mb_loss, frames)."""
    V = _f32(V)
    N, F = V.shape
    W = _f64(W).copy()
    K = W.shape[0]
    A = np.zeros((K, F)) if A is None else _f64(A).copy()
    B = np.zeros((K, F)) if B is None else _f64(B).copy()
    H = np.zeros((N, K)) if want_H else None
    Hi = None if H_init is None else _f64(H_init)
    nmb = (N + beta - 1) // beta
    mb = np.zeros(max(nmb, 1))
    ls = ctypes.c_double(loss_sum)
    done = _lib().or_online_pass(F, K, N, _ptr(V), F, beta, n_in, eps, gamma, r,
                                 n_ref, int(normalize), int(rho_on_new),
                                 int(flush), h_penalty, h_penalty_a, w_penalty,
                                 _ptr(W), _ptr(A), _ptr(B), _ptr(Hi),
                                 _ptr(H), ctypes.byref(ls), _ptr(mb))
    nmb_done = (done + beta - 1) // beta if flush else done // beta
    return dict(W=W, A=A, B=B, H=H, loss_sum=ls.value, mb_loss=mb[:nmb_done],
                frames=done)


def project(V, W, eps=1e-12, gamma=0.5, n_in=10, h_penalty=0.0, h_penalty_a=1.0):
    """h-solve of every frame with W fixed (penalized as in online_pass).
    Returns (H (N,K), obj_sum) with obj_sum the d_IS part."""
    V = _f32(V)
    W = _f64(W)
    N, F = V.shape
    K = W.shape[0]
    H = np.zeros((N, K))
    s = ctypes.c_double(0.0)
    _lib().or_project(F, K, N, _ptr(V), F, _ptr(W), eps, gamma, n_in, h_penalty,
                      h_penalty_a, _ptr(H), ctypes.byref(s))
    return H, s.value


def batch_h0(V, W, eps=1e-12):
    V = _f32(V)
    W = _f64(W)
    N, F = V.shape
    K = W.shape[0]
    H = np.zeros((N, K))
    _lib().or_batch_h0(F, K, N, _ptr(V), F, _ptr(W), eps, _ptr(H))
    return H


def batch(V, W, H, eps=1e-12, gamma=0.5, n_iter=1, normalize=True, which=0):
    """Batch IS-NMF iterations. Returns (W, H, obj (n_iter,))."""
    V = _f32(V)
    W = _f64(W).copy()
    H = _f64(H).copy()
    N, F = V.shape
    K = W.shape[0]
    obj = np.zeros(max(n_iter, 1))
    _lib().or_batch(F, K, N, _ptr(V), F, _ptr(W), _ptr(H), eps, gamma, n_iter,
                    int(normalize), _ptr(obj), int(which))
    return W, H, obj[:n_iter]
