"""Penalized online IS-NMF (Section 2.2, "Extensions") through the C ABI,
against the FP64 oracle: the h penalty lambda * log(a + sum_k h_k) (tangent
majorization in the h update) and the dictionary penalty mu * sum W
(W = sqrt(A/(B + mu))). Element-wise (helpers.parity; rows of W, A, B
including the last): FP32 path 1e-5 on W, A, B, H and the loss; the mma and
cluster h-solves of the mixed path the one-minibatch bounds
(test_gpu_online.MIXED_TOL) and 1e-3 on the loss. The unpenalized mma kernels
are separate instantiations; the cluster kernels take the penalty at run
time (a zero penalty gives the plain kernel's bits)."""
import numpy as np
import pytest

import oracle
import paper_1106_4198_gb300 as onmf
from helpers import cuda, parity, problem, relerr
from test_gpu_online import MIXED_TOL, compare, run_gpu

pytestmark = pytest.mark.gpu
FP32 = onmf.ONMF_FP32


def oracle_pass(V, W0, beta, n_in, **kw):
    oracle.set_threads(16)
    o = oracle.online_pass(V, W0, beta=beta, n_in=n_in, **kw)
    oracle.set_threads(1)
    return o


@pytest.mark.parametrize("F,K,N,beta,n_in", [(129, 8, 2000, 50, 5), (513, 100, 1000, 1000, 10),
                                             (65, 200, 96, 32, 3)])
@pytest.mark.parametrize("lam,a,mu", [(0.5, 1.0, 0.0), (0.0, 1.0, 0.2), (4.0, 0.3, 0.05)])
def test_penalized_pass_matches_oracle(F, K, N, beta, n_in, lam, a, mu):
    """Includes K = 200 (two 128-wide k blocks of the FP32 h update, whose
    penalty uses the frame sums taken before either block is updated)."""
    V, W0 = problem(F, K, N, seed=41 + K)
    pen = dict(h_penalty=lam, h_penalty_a=a, w_penalty=mu)
    g = run_gpu(V, W0, beta=beta, n_inner=n_in, precision=FP32, **pen)
    o = oracle_pass(V, W0, beta, n_in, **pen)
    compare(g, o, 1e-5, label="penalized FP32 F=%d K=%d lam=%g a=%g mu=%g" % (F, K, lam, a, mu))


def test_penalized_projection_matches_oracle():
    F, K, N = 257, 24, 300
    V, W0 = problem(F, K, N, seed=45)
    lam, a = 2.0, 0.5
    m = onmf.OnlineISNMF(F, K, W0, precision=FP32, h_penalty=lam, h_penalty_a=a)
    import torch
    H = torch.empty((N, K), device="cuda")
    m.project(cuda(V), H, n_inner=8)
    m.close()
    Ho, _ = oracle.project(V, W0, n_in=8, h_penalty=lam, h_penalty_a=a)
    parity("penalized projection FP32", dict(H=(H.cpu().numpy(), Ho)), 1e-5)


def test_h_penalty_shrinks_activations_on_gpu():
    F, K, N = 129, 8, 400
    V, W0 = problem(F, K, N, seed=46)
    sums = []
    for lam in (0.0, 2.0, 20.0):
        g = run_gpu(V, W0, beta=50, n_inner=5, precision=FP32, h_penalty=lam)
        sums.append(float(g["H"].sum()))
    assert sums[0] > sums[1] > sums[2], sums


@pytest.mark.parametrize("F,K,N,beta,n_in", [(129, 8, 2000, 50, 5), (513, 100, 1000, 1000, 10),
                                             (65, 128, 96, 32, 3)])
@pytest.mark.parametrize("lam,a,mu", [(0.5, 1.0, 0.0), (4.0, 0.3, 0.05)])
def test_penalized_pass_mixed_mma(F, K, N, beta, n_in, lam, a, mu):
    V, W0 = problem(F, K, N, seed=51 + K)
    pen = dict(h_penalty=lam, h_penalty_a=a, w_penalty=mu)
    g = run_gpu(V, W0, beta=beta, n_inner=n_in, precision=onmf.ONMF_MIXED,
                hsolve=onmf.ONMF_HSOLVE_MMA, **pen)
    o = oracle_pass(V, W0, beta, n_in, **pen)
    compare(g, o, MIXED_TOL, label="penalized mixed F=%d K=%d lam=%g a=%g mu=%g"
            % (F, K, lam, a, mu))
    # the activations follow the penalized oracle, not the unpenalized one
    # (W moves by less than the bf16 error here, H by more)
    ou = oracle_pass(V, W0, beta, n_in)
    assert relerr(g["H"], o["H"]) < relerr(g["H"], ou["H"])


def test_penalized_projection_mixed_mma():
    import torch
    F, K, N = 257, 24, 300
    V, W0 = problem(F, K, N, seed=55)
    lam, a = 2.0, 0.5
    m = onmf.OnlineISNMF(F, K, W0, precision=onmf.ONMF_MIXED, hsolve=onmf.ONMF_HSOLVE_MMA,
                         h_penalty=lam, h_penalty_a=a)
    H = torch.empty((N, K), device="cuda")
    m.project(cuda(V), H, n_inner=8)
    m.close()
    Ho, _ = oracle.project(V, W0, n_in=8, h_penalty=lam, h_penalty_a=a)
    parity("penalized projection mixed", dict(H=(H.cpu().numpy(), Ho)), MIXED_TOL["H"])


@pytest.mark.parametrize("F,K,N,beta,n_in", [(129, 8, 512, 64, 5), (513, 100, 1000, 500, 6),
                                             (257, 256, 256, 128, 4)])
@pytest.mark.parametrize("lam,a,mu", [(0.5, 1.0, 0.0), (4.0, 0.3, 0.05)])
def test_penalized_pass_mixed_cluster(F, K, N, beta, n_in, lam, a, mu):
    """The cluster h-solve (the only one for K > 128): the h penalty in the
    owners' update (frame sums over all k before the step), the dictionary
    penalty in the statistics epilogue."""
    V, W0 = problem(F, K, N, seed=61 + K)
    pen = dict(h_penalty=lam, h_penalty_a=a, w_penalty=mu)
    g = run_gpu(V, W0, beta=beta, n_inner=n_in, precision=onmf.ONMF_MIXED,
                hsolve=onmf.ONMF_HSOLVE_CLUSTER, **pen)
    o = oracle_pass(V, W0, beta, n_in, **pen)
    compare(g, o, MIXED_TOL, label="penalized mixed cluster F=%d K=%d lam=%g a=%g mu=%g"
            % (F, K, lam, a, mu))
    ou = oracle_pass(V, W0, beta, n_in)
    assert relerr(g["H"], o["H"]) < relerr(g["H"], ou["H"])


def test_zero_penalty_cluster_is_the_plain_kernel():
    """With lambda = mu = 0 the cluster kernels take their plain path: the
    same bits as a run without penalties."""
    V, W0 = problem(257, 160, 256, seed=67)
    a = run_gpu(V, W0, beta=128, n_inner=4, precision=onmf.ONMF_MIXED,
                hsolve=onmf.ONMF_HSOLVE_CLUSTER)
    b = run_gpu(V, W0, beta=128, n_inner=4, precision=onmf.ONMF_MIXED,
                hsolve=onmf.ONMF_HSOLVE_CLUSTER, h_penalty=0.0, w_penalty=0.0)
    assert np.array_equal(a["W"], b["W"]) and np.array_equal(a["H"], b["H"])


def test_penalized_projection_mixed_cluster():
    import torch
    F, K, N = 257, 160, 300
    V, W0 = problem(F, K, N, seed=69)
    lam, a = 2.0, 0.5
    m = onmf.OnlineISNMF(F, K, W0, precision=onmf.ONMF_MIXED, hsolve=onmf.ONMF_HSOLVE_CLUSTER,
                         h_penalty=lam, h_penalty_a=a)
    H = torch.empty((N, K), device="cuda")
    m.project(cuda(V), H, n_inner=8)
    m.close()
    Ho, _ = oracle.project(V, W0, n_in=8, h_penalty=lam, h_penalty_a=a)
    parity("penalized projection mixed cluster", dict(H=(H.cpu().numpy(), Ho)), MIXED_TOL["H"])
