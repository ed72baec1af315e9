"""Parity of the online IS-NMF step (Algorithm 1) on the GPU, called through
the C ABI, against the FP64 oracle on the same seeded inputs.

Every comparison is element-wise (helpers.parity): each entry within
tol * (|x_ref| + 1e-3 mean|x_ref|), and for W, A, B each frequency row within
tol in norm, the last row f = F - 1 asserted on its own.
  FP32, one minibatch:          W, H, A, B and the loss <= 1e-5
  FP32, objective trajectory:   every minibatch loss <= 1e-3 (up to 100 steps)
  mixed (BF16 products):        MIXED_TOL, about three times the largest
                                error measured on a GB300 (printed by the test)
"""
import numpy as np
import pytest

import oracle
import paper_1106_4198_gb300 as onmf
from helpers import cuda, parity, problem

pytestmark = pytest.mark.gpu

FP32 = onmf.ONMF_FP32
MIXED = onmf.ONMF_MIXED


def run_gpu(V, W0, chunks=None, flush=True, want_H=True, device_input=True, **cfg):
    """Push V (in `chunks` pieces) through one state; return its outputs."""
    import torch
    K, F = W0.shape
    N = V.shape[0]
    m = onmf.OnlineISNMF(F, K, W0, **cfg)
    Vd = cuda(V) if device_input else np.ascontiguousarray(V)
    H = torch.zeros((N, K), device="cuda") if want_H else None
    bounds = [0] + list(np.cumsum(chunks if chunks else [N]))
    for a, b in zip(bounds[:-1], bounds[1:]):
        m.push(Vd[a:b], H[a:b] if want_H else None)
    if flush:
        m.flush()
    m.sync()
    W = m.W()
    A, B, t, ls = m.stats()
    out = dict(W=W, A=A, B=B, t=t, loss_sum=ls,
               H=H.cpu().numpy() if want_H else None)
    m.close()
    return out


def run_oracle(V, W0, beta, n_inner, eps=1e-12, r=1.0, n_ref=0, h_exponent=0.5,
               normalize=1, rho_on_new=0, flush=True):
    oracle.set_threads(16)
    o = oracle.online_pass(V, W0, beta=beta, n_in=n_inner, eps=eps,
                           gamma=h_exponent, r=r, n_ref=n_ref,
                           normalize=bool(normalize),
                           rho_on_new=bool(rho_on_new), flush=flush)
    oracle.set_threads(1)
    return o


# Element-wise bounds of the mixed path (BF16 operands of the products,
# FP32 ratios, FP64 or compensated A and B) for one minibatch: about three
# times the largest error measured on a GB300 over the one-minibatch, warm,
# penalty, accumulator and cluster tests (W 1.4e-3, A 5.5e-3, B 2.8e-3,
# H 3.0e-3 per entry; loss 2.2e-5).
MIXED_TOL = dict(W=4e-3, A=1.6e-2, B=9e-3, H=9e-3, loss=1e-4)


def pairs_of(g, o, nframes=None):
    """(GPU, oracle) pairs of one run's outputs."""
    p = dict(W=(g["W"], o["W"]), A=(g["A"], o["A"]), B=(g["B"], o["B"]))
    if g["H"] is not None:
        n = nframes if nframes is not None else o["frames"]
        p["H"] = (g["H"][:n], o["H"][:n])
    p["loss"] = (g["loss_sum"], o["loss_sum"])
    return p


def compare(g, o, tol, nframes=None, label="online"):
    return parity(label, pairs_of(g, o, nframes), tol)


@pytest.mark.parametrize("F,K,beta,n_in", [(129, 8, 50, 5), (513, 100, 1000, 10),
                                           (17, 3, 13, 4), (40, 33, 24, 3)])
def test_fp32_single_minibatch(F, K, beta, n_in):
    V, W0 = problem(F, K, beta)
    g = run_gpu(V, W0, beta=beta, n_inner=n_in, precision=FP32)
    o = run_oracle(V, W0, beta, n_in)
    assert g["t"] == beta
    compare(g, o, 1e-5)


def test_fp32_c1_pass_objective_trajectory():
    """Config 1 shape: F=129, K=8, N=2000, beta=50, 5 inner steps, one pass.
    Every minibatch's loss within 1e-3 of the oracle's."""
    F, K, N, beta, n_in = 129, 8, 2000, 50, 5
    V, W0 = problem(F, K, N)
    o = run_oracle(V, W0, beta, n_in)
    # per-minibatch losses from the running sum, one minibatch per push
    m = onmf.OnlineISNMF(F, K, W0, beta=beta, n_inner=n_in, precision=FP32)
    Vd = cuda(V)
    prev = 0.0
    worst = 0.0
    for i in range(N // beta):
        m.push(Vd[i * beta:(i + 1) * beta])
        _, _, _, ls = m.stats()
        lg = ls - prev
        prev = ls
        worst = max(worst, abs(lg - o["mb_loss"][i]) / abs(o["mb_loss"][i]))
    W = m.W()
    A, B, _, _ = m.stats()
    m.close()
    print("worst minibatch loss rel err %.2e" % worst)
    assert worst <= 1e-3
    parity("C1 pass FP32", dict(W=(W, o["W"]), A=(A, o["A"]), B=(B, o["B"])), 1e-5)


def test_ragged_pushes_and_flush():
    """beta not a multiple of the 8-frame tile, pushes that straddle
    minibatches, and a partial last minibatch processed by flush."""
    F, K, beta, n_in = 17, 3, 13, 4
    V, W0 = problem(F, K, 45)
    g = run_gpu(V, W0, chunks=[5, 20, 1, 19], beta=beta, n_inner=n_in,
                precision=FP32, r=0.7, n_ref=45)
    o = run_oracle(V, W0, beta, n_in, r=0.7, n_ref=45)
    assert g["t"] == 45
    compare(g, o, 1e-5)


def test_split_push_is_bitwise_identical():
    """The minibatches, not the push boundaries, define the computation."""
    F, K, beta = 129, 8, 50
    V, W0 = problem(F, K, 400)
    a = run_gpu(V, W0, beta=beta, n_inner=5)
    b = run_gpu(V, W0, chunks=[7, 93, 150, 1, 149], beta=beta, n_inner=5)
    assert np.array_equal(a["W"], b["W"]) and np.array_equal(a["A"], b["A"])
    assert np.array_equal(a["H"], b["H"]) and a["loss_sum"] == b["loss_sum"]


def test_host_input_matches_device_input():
    F, K, beta = 129, 8, 50
    V, W0 = problem(F, K, 300)
    a = run_gpu(V, W0, beta=beta, n_inner=5)
    b = run_gpu(V, W0, beta=beta, n_inner=5, device_input=False)
    assert np.array_equal(a["W"], b["W"]) and np.array_equal(a["H"], b["H"])


def test_host_input_ring_crosses_slots():
    """Host frames run through a two-slot device ring filled on a copy stream.
    beta = 2**18 makes one slot hold exactly one minibatch, so 2.5 minibatches
    reuse both slots and leave a ragged tail in staging. Pageable, page-locked
    (pulled by a copy kernel) and strided host buffers (with host H_out) all
    equal the device path."""
    import torch
    F, K, beta = 33, 4, 1 << 18
    N = 5 * beta // 2
    V, W0 = problem(F, K, N, seed=11)
    ref = run_gpu(V, W0, beta=beta, n_inner=3, precision=MIXED)
    pinned = torch.from_numpy(V).pin_memory()
    wide = np.zeros((N, F + 3), dtype=np.float32)
    wide[:, :F] = V
    wide_pinned = torch.from_numpy(wide).pin_memory()[:, :F]  # strided, page-locked
    for Vh in (np.ascontiguousarray(V), pinned, wide[:, :F], wide_pinned):
        m = onmf.OnlineISNMF(F, K, W0, beta=beta, n_inner=3, precision=MIXED)
        H = np.zeros((N, K), dtype=np.float32)
        m.push(Vh, H)
        m.flush()
        m.sync()
        assert np.array_equal(m.W(), ref["W"])
        assert np.array_equal(H, ref["H"])
        m.close()


def test_scale_equivariance_bitwise_gpu(hsolve):
    """eps = 0: V -> 4V leaves W, A, B bit-identical and scales H by 4
    (power-of-two scaling is exact and every ratio is invariant)."""
    F, K, beta = 129, 8, 50
    V, W0 = problem(F, K, 200)
    for prec in (FP32, MIXED):
        a = run_gpu(V, W0, beta=beta, n_inner=5, eps=0.0, precision=prec)
        b = run_gpu(4 * V, W0, beta=beta, n_inner=5, eps=0.0, precision=prec)
        assert np.array_equal(a["W"], b["W"]), prec
        assert np.array_equal(a["A"], b["A"]) and np.array_equal(a["B"], b["B"])
        assert np.array_equal(4 * a["H"], b["H"])


def test_checkpoint_resume_bitwise():
    F, K, beta = 129, 8, 50
    V, W0 = problem(F, K, 400)
    full = run_gpu(V, W0, beta=beta, n_inner=5, want_H=False)
    m = onmf.OnlineISNMF(F, K, W0, beta=beta, n_inner=5)
    m.push(cuda(V[:200]))
    W = m.W()
    A, B, t, ls = m.stats()
    m.close()
    m2 = onmf.OnlineISNMF(F, K, W0, beta=beta, n_inner=5)
    m2.set_state(W, A, B, t, ls)
    m2.push(cuda(V[200:]))
    W2 = m2.W()
    A2, B2, t2, ls2 = m2.stats()
    m2.close()
    assert t2 == 400
    assert np.array_equal(W2, full["W"]) and np.array_equal(A2, full["A"])
    assert ls2 == full["loss_sum"]


@pytest.mark.parametrize("precision", [FP32, MIXED])
def test_invalid_frames_are_reported_and_sticky(precision):
    """A NaN or a negative frame value: ONMF_ENUMERIC at the next sync, then
    ONMF_ESTATE until the state is set again. On the mixed path the check
    runs while the frames are staged, inside the previous minibatch's grid
    barrier window; the CTA that saw it carries the error to its next grid
    barrier, where every CTA leaves the kernel."""
    F, K, beta = 33, 4, 16
    V, W0 = problem(F, K, 48)
    V = V.copy()
    V[20, 5] = np.nan
    m = onmf.OnlineISNMF(F, K, W0, beta=beta, n_inner=3, precision=precision)
    m.push(cuda(V))
    with pytest.raises(onmf.OnmfError) as e:
        m.sync()
    assert e.value.status == 5  # ONMF_ENUMERIC
    with pytest.raises(onmf.OnmfError) as e:
        m.push(cuda(V[:16]))
    assert e.value.status == 7  # ONMF_ESTATE (sticky)
    # the first minibatch (frames 0..15) was applied, the bad one was not
    o = run_oracle(V[:16], W0, beta, 3)
    m.set_state(o["W"].astype(np.float32), o["A"], o["B"], 16, o["loss_sum"])
    m.push(cuda(V[32:48]))
    m.sync()
    m.close()
    V[20, 5] = -1.0
    m = onmf.OnlineISNMF(F, K, W0, beta=beta, n_inner=3, precision=precision)
    m.push(cuda(V))
    with pytest.raises(onmf.OnmfError):
        m.sync()
    m.close()


def test_projection_fp32():
    F, K, n = 513, 100, 300
    V, W0 = problem(F, K, n)
    m = onmf.OnlineISNMF(F, K, W0, n_inner=10)
    import torch
    H = torch.zeros((n, K), device="cuda")
    obj = m.project(cuda(V), H, want_obj=True)
    m.close()
    oracle.set_threads(16)
    Ho, so = oracle.project(V, W0, n_in=10)
    oracle.set_threads(1)
    parity("projection FP32", dict(H=(H.cpu().numpy(), Ho), objective=(obj, so)), 1e-5)


def test_projection_block_diagonal_closed_form():
    """F = 513, K = 100, eps = 0, disjoint row supports per column: every h_k
    follows the K = 1 closed form log h_k(n) = log h*_k + (log h0 - log h*_k)/2^n."""
    import torch
    F, K, n_in, n = 513, 100, 10, 16
    r = np.random.default_rng(4)
    owner = np.arange(F) % K
    W = np.zeros((K, F), dtype=np.float32)
    W[owner, np.arange(F)] = r.gamma(1.0, 1.0, F) + 0.05
    V = (r.gamma(1.0, 1.0, (n, F)) + 0.05).astype(np.float32)
    m = onmf.OnlineISNMF(F, K, W, n_inner=n_in, eps=0.0)
    H = torch.zeros((n, K), device="cuda")
    m.project(cuda(V), H)
    m.close()
    H = H.cpu().numpy().astype(np.float64)
    Wd = W.astype(np.float64)
    worst = 0.0
    for j in range(n):
        h0 = V[j].astype(np.float64).sum() / Wd.sum()
        for k in range(K):
            sel = owner == k
            hs = np.mean(V[j, sel].astype(np.float64) / Wd[k, sel])
            expect = np.exp(np.log(hs) + (np.log(h0) - np.log(hs)) / 2 ** n_in)
            worst = max(worst, abs(H[j, k] - expect) / expect)
    print("closed-form worst rel err %.2e" % worst)
    assert worst <= 1e-5


@pytest.fixture(params=["mma", "tc", "cluster"])
def hsolve(request, monkeypatch):
    """Mixed precision has three h-solves: mma.sync on one CTA per 8-frame
    tile (default for K <= 128), tcgen05 (ONMF_HSOLVE=tc) and the cluster
    h-solve (ONMF_HSOLVE=cluster; always for K > 128); every mixed test runs
    on each."""
    monkeypatch.setenv("ONMF_HSOLVE", request.param)
    return request.param


@pytest.mark.parametrize("F,K,beta,n_in", [(129, 8, 50, 5), (513, 100, 1000, 10),
                                           (513, 128, 512, 10), (256, 40, 37, 4)])
def test_mixed_single_minibatch_error_stated(F, K, beta, n_in, hsolve):
    """Mixed precision (BF16 tensor-core products, FP32 ratios, FP64 A/B):
    one minibatch against the FP64 oracle, element-wise within MIXED_TOL
    (rows of W, A, B including the last one), the minibatch loss within 1e-3."""
    V, W0 = problem(F, K, beta)
    g = run_gpu(V, W0, beta=beta, n_inner=n_in, precision=MIXED)
    o = run_oracle(V, W0, beta, n_in)
    compare(g, o, MIXED_TOL, label="mixed %s F=%d K=%d beta=%d" % (hsolve, F, K, beta))
