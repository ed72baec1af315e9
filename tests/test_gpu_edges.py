"""Degenerate and extreme shapes through the C ABI against the FP64 oracle,
for every h-solve kernel that takes the shape: F = 1, K = 1, beta = 1,
n_inner = 0 (the statistics of the start point alone), gamma = 1 (the
heuristic multiplicative update), F = 1024 with K = 256 (the largest mixed
shape), and empty pushes. Element-wise (helpers.parity, rows of W, A, B
including the last): FP32 within 1e-5; mixed within EDGE_TOL below; the loss
within 1e-5 (FP32) or 1e-3 (mixed) relative, with an absolute slack where it
is about zero."""
import numpy as np
import pytest

import paper_1106_4198_gb300 as onmf
from helpers import parity, problem
from test_gpu_online import run_gpu, run_oracle

pytestmark = pytest.mark.gpu
# Mixed bounds of the degenerate shapes (K = 1, F = 1, 16, 17, single-frame
# minibatches, no inner iterations): about three times the largest measured
# (W 4.1e-3, A 7.2e-3, B 4.8e-3, H 6.5e-3 per entry).
EDGE_TOL = dict(W=1.2e-2, A=2.2e-2, B=1.5e-2, H=2e-2)
FP32, MIXED = onmf.ONMF_FP32, onmf.ONMF_MIXED

KERNELS = [(FP32, 0), (MIXED, onmf.ONMF_HSOLVE_MMA), (MIXED, onmf.ONMF_HSOLVE_TC),
           (MIXED, onmf.ONMF_HSOLVE_CLUSTER)]


def allowed(F, K, precision, hsolve):
    if precision == FP32:
        return True
    if F > 1024 or (hsolve in (onmf.ONMF_HSOLVE_MMA, onmf.ONMF_HSOLVE_TC) and K > 128):
        return False
    if hsolve == onmf.ONMF_HSOLVE_TC:
        tail = F % 128
        return F >= 128 and tail <= 32
    return True


def check(F, K, N, beta, n_in, precision, hsolve, chunks=None, **kw):
    if not allowed(F, K, precision, hsolve):
        pytest.skip("kernel does not take F=%d K=%d" % (F, K))
    V, W0 = problem(F, K, N, seed=81 + F + K)
    try:
        g = run_gpu(V, W0, chunks=chunks, beta=beta, n_inner=n_in, precision=precision,
                    hsolve=hsolve, **kw)
    except onmf.OnmfError as err:
        if err.status == 1:  # the library does not offer this kernel for the shape
            pytest.skip(str(err))
        raise
    o = run_oracle(V, W0, beta, n_in, **{k: v for k, v in kw.items() if k != "hsolve"})
    # the loss can be ~0 (F = K = 1: the start point is already exact), where
    # a relative error means nothing; the absolute slack is the per-bin d_IS
    # of the rounding: FP32 cancellation in (r - 1) - log r (~1e-11), or
    # (delta^2)/2 with delta = 2^-9 for the bf16 h of the mixed path
    tol_l = 1e-5 if precision == FP32 else 1e-3
    tol = 1e-5 if precision == FP32 else EDGE_TOL
    per_bin = 1e-10 if precision == FP32 else 1e-5
    dl = abs(g["loss_sum"] - o["loss_sum"])
    eloss = dl / (tol_l * abs(o["loss_sum"]) + per_bin * F * N) * tol_l
    label = "F=%d K=%d N=%d beta=%d n_in=%d prec=%d hsolve=%d" % (F, K, N, beta, n_in,
                                                                   precision, hsolve)
    print("%s: loss %.1e" % (label, eloss))
    assert g["t"] == N
    assert eloss <= tol_l
    parity(label, dict(W=(g["W"], o["W"]), A=(g["A"], o["A"]), B=(g["B"], o["B"]),
                       H=(g["H"], o["H"])), tol)


@pytest.mark.parametrize("precision,hsolve", KERNELS)
@pytest.mark.parametrize("F,K", [(1, 1), (17, 1), (16, 16), (130, 3)])
def test_tiny_shapes(F, K, precision, hsolve):
    check(F, K, 40, 13, 3, precision, hsolve, chunks=[1, 12, 27])


@pytest.mark.parametrize("precision,hsolve", KERNELS)
def test_single_frame_minibatches(precision, hsolve):
    check(129, 8, 20, 1, 4, precision, hsolve)


@pytest.mark.parametrize("precision,hsolve", KERNELS)
def test_no_inner_iterations(precision, hsolve):
    """n_inner = 0: every frame keeps its start point; only the statistics
    and the dictionary step run."""
    check(129, 8, 100, 50, 0, precision, hsolve)


@pytest.mark.parametrize("precision,hsolve", KERNELS)
def test_heuristic_exponent(precision, hsolve):
    check(129, 8, 100, 50, 5, precision, hsolve, h_exponent=1.0)


@pytest.mark.parametrize("precision,hsolve", [(FP32, 0), (MIXED, onmf.ONMF_HSOLVE_CLUSTER)])
def test_largest_mixed_shape(precision, hsolve):
    check(1024, 256, 300, 256, 4, precision, hsolve)


def test_empty_pushes_change_nothing():
    import torch
    F, K = 65, 4
    V, W0 = problem(F, K, 10, seed=90)
    for hs in (0, onmf.ONMF_HSOLVE_CLUSTER):
        m = onmf.OnlineISNMF(F, K, W0, beta=4, n_inner=2, precision=MIXED, hsolve=hs)
        m.push(torch.zeros((0, F), device="cuda"))
        m.flush()
        m.sync()
        assert np.array_equal(m.W(), W0.astype(np.float32))
        _, _, t, ls = m.stats()
        assert t == 0 and ls == 0.0
        m.close()
