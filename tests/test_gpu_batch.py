"""Parity of batch IS-NMF multiplicative updates (Section 2.1) on the GPU,
through the C ABI (nmf_batch_init_H, nmf_batch_step), against the FP64 oracle.

Tolerances: FP32 one cycle W, H element-wise <= 1e-5 (helpers.parity: every
entry, and every frequency row of W including the last); objective
trajectory <= 1e-3 at every cycle (50 cycles, config-1 shape); mixed
precision stated per test. A batch plan (nmf_batch_plan_*) gives the same
bits as the one-shot call and allocates nothing per call."""
import numpy as np
import pytest

import oracle
import paper_1106_4198_gb300 as onmf
from helpers import cuda, parity, problem, relerr

pytestmark = pytest.mark.gpu


def gpu_batch(V, W0, n_iter, precision=onmf.ONMF_FP32, eps=1e-12, H0=None):
    import torch
    K, F = W0.shape
    N = V.shape[0]
    Vd = cuda(V)
    W = cuda(W0.astype(np.float32))
    if H0 is None:
        H = torch.zeros((N, K), device="cuda")
        onmf.nmf_batch_init_H(Vd, W, H, eps=eps)
    else:
        H = cuda(H0.astype(np.float32))
    obj = onmf.nmf_batch_step(Vd, W, H, eps=eps, n_iter=n_iter, precision=precision)
    torch.cuda.synchronize()
    return W.cpu().numpy(), H.cpu().numpy(), obj


def test_batch_start_point():
    import torch
    F, K, N = 129, 8, 500
    V, W0 = problem(F, K, N)
    H = torch.zeros((N, K), device="cuda")
    onmf.nmf_batch_init_H(cuda(V), cuda(W0), H, eps=1e-12)
    Ho = oracle.batch_h0(V, W0, eps=1e-12)
    assert relerr(H.cpu().numpy(), Ho) <= 1e-6


@pytest.mark.parametrize("F,K,N", [(129, 8, 2000), (513, 50, 3000), (33, 5, 41)])
def test_batch_one_cycle_fp32(F, K, N):
    V, W0 = problem(F, K, N)
    H0 = oracle.batch_h0(V, W0)
    Wg, Hg, objg = gpu_batch(V, W0, 1, H0=H0)
    oracle.set_threads(16)
    Wo, Ho, objo = oracle.batch(V, W0, H0, n_iter=1)
    oracle.set_threads(1)
    parity("batch one cycle F=%d K=%d N=%d" % (F, K, N),
           dict(W=(Wg, Wo), H=(Hg, Ho), objective=(objg[0], objo[0])), 1e-5)


def test_batch_c1_objective_trajectory():
    """Config 1: F=129, K=8, N=2000, 50 cycles; every cycle's objective
    within 1e-3 of the oracle, and (FP32) non-increasing."""
    F, K, N, it = 129, 8, 2000, 50
    V, W0 = problem(F, K, N)
    H0 = oracle.batch_h0(V, W0)
    Wg, Hg, objg = gpu_batch(V, W0, it, H0=H0)
    oracle.set_threads(16)
    Wo, Ho, objo = oracle.batch(V, W0, H0, n_iter=it)
    oracle.set_threads(1)
    rel = np.abs(objg - objo) / objo
    print("batch C1: worst objective rel err %.2e" % rel.max())
    assert rel.max() <= 1e-3
    assert np.all(np.diff(objg) <= 1e-6 * objg[:-1])
    parity("batch C1 50 cycles FP32", dict(W=(Wg, Wo), H=(Hg, Ho)), 1e-5)


@pytest.mark.parametrize("hsolve", ["mma", "tc"])
def test_batch_mixed_objective_stated(hsolve, monkeypatch):
    """Mixed precision batch cycles (BF16 products, both h-solves): objective
    within 1e-3 of the FP64 oracle at every cycle (config-1 shape, 50 cycles)."""
    if hsolve == "tc":
        monkeypatch.setenv("ONMF_HSOLVE", "tc")
    else:
        monkeypatch.delenv("ONMF_HSOLVE", raising=False)
    F, K, N, it = 129, 8, 2000, 50
    V, W0 = problem(F, K, N)
    H0 = oracle.batch_h0(V, W0)
    _, _, objg = gpu_batch(V, W0, it, precision=onmf.ONMF_MIXED, H0=H0)
    _, _, objo = oracle.batch(V, W0, H0, n_iter=it)
    rel = np.abs(objg - objo) / objo
    print("batch mixed C1: worst objective rel err %.2e" % rel.max())
    assert rel.max() <= 1e-3


@pytest.mark.parametrize("precision,tol", [(onmf.ONMF_FP32, 1e-5), (onmf.ONMF_MIXED, 1e-5)])
@pytest.mark.parametrize("F,K,N", [(129, 8, 2000), (513, 50, 3000)])
def test_online_step_over_all_frames_is_a_batch_cycle(F, K, N, precision, tol):
    """Section 2.3 ("Overview"): with beta = N, r = 0 and one h update from
    the fresh-restart point, one online minibatch is one batch cycle from the
    batch start point (the same h update, then W = sqrt(A/B) =
    W o sqrt((P H^T)/(Q H^T)), then the column rescale). The two GPU paths
    (different kernels and summation orders) give the same W: both round
    the same operands to bf16, so even the mixed path agrees to FP32
    summation order (measured 4.8e-7 per entry)."""
    from test_gpu_online import run_gpu
    V, W0 = problem(F, K, N, seed=K)
    on = run_gpu(V, W0, beta=N, n_inner=1, precision=precision, r=0.0, n_ref=N)
    Wb, _, _ = gpu_batch(V, W0, 1, precision=precision)
    assert on["t"] == N
    parity("online step = batch cycle F=%d K=%d prec=%d" % (F, K, precision),
           dict(W=(on["W"], Wb)), tol)


@pytest.mark.parametrize("precision", [onmf.ONMF_FP32, onmf.ONMF_MIXED])
def test_batch_plan_equals_one_shot_and_allocates_nothing(precision):
    """nmf_batch_plan_step runs the cycles of nmf_batch_step on scratch made
    once: the same W, H and objectives bit for bit, for N below the plan's
    N_max too, and free device memory unchanged across a call after the
    first."""
    import torch
    F, K, N, it = 129, 8, 2000, 6
    V, W0 = problem(F, K, N, seed=21)
    H0 = oracle.batch_h0(V, W0)
    Vd = cuda(V)
    plan = onmf.BatchPlan(F, K, N + 777, precision)
    for n in (N, N - 333):
        W1, H1 = cuda(W0.astype(np.float32)), cuda(H0[:n].astype(np.float32))
        o1 = onmf.nmf_batch_step(Vd[:n], W1, H1, n_iter=it, precision=precision)
        W2, H2 = cuda(W0.astype(np.float32)), cuda(H0[:n].astype(np.float32))
        o2 = plan.step(Vd[:n], W2, H2, n_iter=it)
        torch.cuda.synchronize()
        assert np.array_equal(W1.cpu().numpy(), W2.cpu().numpy())
        assert np.array_equal(H1.cpu().numpy(), H2.cpu().numpy())
        assert np.array_equal(o1, o2)
    W3, H3 = cuda(W0.astype(np.float32)), cuda(H0.astype(np.float32))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    plan.step(Vd, W3, H3, n_iter=it, want_obj=False)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, free0 - free1
    with pytest.raises(onmf.OnmfError):  # more frames than the plan holds
        plan.step(cuda(np.concatenate([V, V])), W3, cuda(np.concatenate([H0, H0])
                                                         .astype(np.float32)), n_iter=1)
    plan.close()
