"""Warm restarts over a finite data set (Section 2.3, "Fresh or warm
restarts", "Finite data sets") through onmf_push_frames_warm (C ABI): each
frame's h-solve starts from its kept activation, frames are visited in a
given order (a new permutation per pass), the final h goes back to its row.

Checked against the FP64 oracle run on the same permuted frames and start
points, element-wise (helpers.parity): FP32 within 1e-5 (W, A, B, H,
loss), mixed within test_gpu_online.MIXED_TOL; the identity order equals no order bit for
bit; fresh and warm frames never share a staged minibatch."""
import numpy as np
import pytest

import oracle
import paper_1106_4198_gb300 as onmf
from helpers import cuda, parity, problem
from test_gpu_online import MIXED_TOL

pytestmark = pytest.mark.gpu
FP32, MIXED = onmf.ONMF_FP32, onmf.ONMF_MIXED


def gpu_passes(V, W0, H0, orders, beta, n_in, precision=FP32, **cfg):
    """Warm passes over V (N, F) with start points H0 (N, K); one push per
    pass in the given order (None: rows in order), then a flush."""
    import torch
    K, F = W0.shape
    m = onmf.OnlineISNMF(F, K, W0, beta=beta, n_inner=n_in, precision=precision, **cfg)
    Vd = cuda(V)
    Hd = cuda(H0.astype(np.float32))
    for o in orders:
        od = None if o is None else torch.as_tensor(o, dtype=torch.int64).cuda()
        m.push_warm(Vd, Hd, od)
        m.flush()
    m.sync()
    W = m.W()
    A, B, t, ls = m.stats()
    m.close()
    return dict(W=W, A=A, B=B, t=t, loss_sum=ls, H=Hd.cpu().numpy())


def oracle_passes(V, W0, H0, orders, beta, n_in, **kw):
    oracle.set_threads(16)
    W, A, B = W0.astype(np.float64), None, None
    H = H0.astype(np.float32).astype(np.float64)
    ls = 0.0
    for o in orders:
        idx = np.arange(V.shape[0]) if o is None else o
        out = oracle.online_pass(V[idx], W, A, B, beta=beta, n_in=n_in, H_init=H[idx],
                                 loss_sum=ls, **kw)
        W, A, B, ls = out["W"], out["A"], out["B"], out["loss_sum"]
        H[idx] = out["H"]
    oracle.set_threads(1)
    return dict(W=W, A=A, B=B, H=H, loss_sum=ls)


def errors(label, g, o, tol):
    return parity(label, dict(W=(g["W"], o["W"]), A=(g["A"], o["A"]), B=(g["B"], o["B"]),
                              H=(g["H"], o["H"]), loss=(g["loss_sum"], o["loss_sum"])), tol)


def start_points(N, K, seed):
    return (np.random.default_rng(seed).gamma(1.0, 1.0, size=(N, K)) * 50 + 1.0).astype(np.float32)


def test_fp32_warm_pass_permuted_ragged():
    """One permuted pass, beta = 50 over 333 frames (6 minibatches and a
    flushed one of 33), two h updates per visit, r = 0.7."""
    F, K, N, beta = 129, 8, 333, 50
    V, W0 = problem(F, K, N, seed=51)
    H0 = start_points(N, K, 52)
    order = np.random.default_rng(53).permutation(N)
    kw = dict(r=0.7, n_ref=N)
    g = gpu_passes(V, W0, H0, [order], beta, 2, **kw)
    o = oracle_passes(V, W0, H0, [order], beta, 2, **kw)
    assert g["t"] == N
    errors("FP32 warm pass", g, o, 1e-5)


def test_fp32_three_warm_passes_with_new_permutations():
    F, K, N, beta = 129, 8, 256, 64
    V, W0 = problem(F, K, N, seed=54)
    H0 = start_points(N, K, 55)
    rng = np.random.default_rng(56)
    orders = [rng.permutation(N) for _ in range(3)]
    g = gpu_passes(V, W0, H0, orders, beta, 1)
    o = oracle_passes(V, W0, H0, orders, beta, 1)
    errors("FP32 three warm passes", g, o, 1e-5)


@pytest.mark.parametrize("hsolve", ["mma", "cluster"])
def test_mixed_warm_pass_error_stated(hsolve, monkeypatch):
    monkeypatch.setenv("ONMF_HSOLVE", hsolve)
    F, K, N, beta = 513, 100, 1200, 500
    V, W0 = problem(F, K, N, seed=57)
    H0 = start_points(N, K, 58)
    order = np.random.default_rng(59).permutation(N)
    g = gpu_passes(V, W0, H0, [order], beta, 3, precision=MIXED)
    o = oracle_passes(V, W0, H0, [order], beta, 3)
    errors("mixed (%s) warm pass" % hsolve, g, o, MIXED_TOL)


def test_identity_order_equals_no_order_bitwise():
    F, K, N, beta = 129, 8, 200, 64
    V, W0 = problem(F, K, N, seed=60)
    H0 = start_points(N, K, 61)
    a = gpu_passes(V, W0, H0, [None], beta, 2)
    b = gpu_passes(V, W0, H0, [np.arange(N)], beta, 2)
    for k in ("W", "A", "B", "H"):
        assert np.array_equal(a[k], b[k]), k
    assert a["loss_sum"] == b["loss_sum"]


def test_fresh_and_warm_frames_do_not_share_a_minibatch():
    import torch
    F, K, beta = 33, 4, 16
    V, W0 = problem(F, K, 20, seed=62)
    m = onmf.OnlineISNMF(F, K, W0, beta=beta, n_inner=2)
    Vd = cuda(V)
    H = torch.ones((20, K), device="cuda")
    m.push(Vd[:5])  # 5 fresh frames staged
    with pytest.raises(onmf.OnmfError) as e:
        m.push_warm(Vd, H)
    assert e.value.status == 7  # ONMF_ESTATE
    m.flush()
    m.push_warm(Vd[:5], H[:5])  # 5 warm frames staged
    with pytest.raises(onmf.OnmfError) as e:
        m.push(Vd[:3])
    assert e.value.status == 7
    m.flush()
    m.sync()
    m.close()
