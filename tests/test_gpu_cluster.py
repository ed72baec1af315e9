"""The cluster h-solve (mixed precision; W split by rows over the CTAs of a
thread-block cluster, partial W^T [p | q] combined in distributed shared
memory in a fixed order), through the C ABI.

  - the mixed-precision settings of the K x beta sweep at F = 513
    (K in {64, 100, 256}, beta in {512, 2048}, 10 inner iterations): one
    minibatch against the FP64 oracle, element-wise within the one-minibatch
    bounds (test_gpu_online.MIXED_TOL; rows of W, A, B including the last),
    the minibatch loss within 1e-3;
  - K = 256 over several minibatches with ragged pushes and a flush;
  - run-to-run, split-push and host-vs-device results are bit-identical;
  - projection and batch cycles at K = 256 against the oracle."""
import numpy as np
import pytest

import oracle
import paper_1106_4198_gb300 as onmf
from helpers import cuda, parity, problem
from test_gpu_online import MIXED_TOL, compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
MIXED = onmf.ONMF_MIXED


@pytest.fixture(autouse=True)
def cluster_env(monkeypatch):
    monkeypatch.setenv("ONMF_HSOLVE", "cluster")


@pytest.mark.parametrize("K", [64, 100, 256])
@pytest.mark.parametrize("beta", [512, 2048])
@pytest.mark.parametrize("hsolve", ["cluster", "mma", "tc"])
def test_sweep_setting_one_minibatch(K, beta, hsolve, monkeypatch):
    """The K x beta sweep at F = 513 on every h-solve kernel that takes the
    shape (mma and tcgen05 stop at K = 128)."""
    if hsolve != "cluster" and K > 128:
        pytest.skip("%s h-solve takes K <= 128" % hsolve)
    monkeypatch.setenv("ONMF_HSOLVE", hsolve)
    F, n_in = 513, 10
    V, W0 = problem(F, K, beta, seed=31)
    g = run_gpu(V, W0, beta=beta, n_inner=n_in, precision=MIXED)
    o = run_oracle(V, W0, beta, n_in)
    compare(g, o, MIXED_TOL, label="sweep F=%d K=%d beta=%d %s" % (F, K, beta, hsolve))


def test_k256_ragged_stream_with_flush():
    F, K, beta, n_in = 513, 256, 300, 6
    N = 1000  # 3 full minibatches and a flushed one of 100
    V, W0 = problem(F, K, N, seed=32)
    g = run_gpu(V, W0, chunks=[1, 299, 17, 450, 233], beta=beta, n_inner=n_in,
                precision=MIXED, r=0.7, n_ref=N)
    o = run_oracle(V, W0, beta, n_in, r=0.7, n_ref=N)
    assert g["t"] == N
    compare(g, o, MIXED_TOL, label="K=256 ragged stream")


@pytest.mark.parametrize("F,K", [(129, 8), (513, 100), (513, 256)])
def test_bitwise_reproducible(F, K):
    """Same inputs twice, the same frames in other push sizes, and host
    frames instead of device frames: identical bits (the cluster reduction
    order is fixed)."""
    V, W0 = problem(F, K, 700, seed=33)
    a = run_gpu(V, W0, beta=256, n_inner=5, precision=MIXED)
    b = run_gpu(V, W0, beta=256, n_inner=5, precision=MIXED)
    c = run_gpu(V, W0, chunks=[3, 300, 1, 396], beta=256, n_inner=5, precision=MIXED)
    d = run_gpu(V, W0, beta=256, n_inner=5, precision=MIXED, device_input=False)
    for x in (b, c, d):
        assert np.array_equal(a["W"], x["W"]) and np.array_equal(a["A"], x["A"])
        assert np.array_equal(a["B"], x["B"]) and np.array_equal(a["H"], x["H"])
        assert a["loss_sum"] == x["loss_sum"]


@pytest.mark.parametrize("F,K,n", [(513, 256, 333), (129, 8, 45)])
def test_projection_against_oracle(F, K, n):
    import torch
    V, W0 = problem(F, K, n, seed=34)
    m = onmf.OnlineISNMF(F, K, W0, n_inner=10, precision=MIXED)
    H = torch.zeros((n, K), device="cuda")
    obj = m.project(cuda(V), H, want_obj=True)
    m.close()
    oracle.set_threads(16)
    Ho, so = oracle.project(V, W0, n_in=10)
    oracle.set_threads(1)
    parity("cluster projection F=%d K=%d n=%d" % (F, K, n),
           dict(H=(H.cpu().numpy(), Ho), objective=(obj, so)),
           dict(H=MIXED_TOL["H"], objective=1e-3))


def test_batch_k256_objective_trajectory():
    import torch
    F, K, N, it = 513, 256, 600, 12
    V, W0 = problem(F, K, N, seed=35)
    H0 = oracle.batch_h0(V, W0)
    W = cuda(W0.astype(np.float32))
    H = cuda(H0.astype(np.float32))
    objg = onmf.nmf_batch_step(cuda(V), W, H, n_iter=it, precision=MIXED)
    torch.cuda.synchronize()
    oracle.set_threads(16)
    _, _, objo = oracle.batch(V, W0, H0, n_iter=it)
    oracle.set_threads(1)
    rel = np.abs(objg - objo) / objo
    print("batch K=256 cluster: worst objective rel err %.2e" % rel.max())
    assert rel.max() <= 1e-3
