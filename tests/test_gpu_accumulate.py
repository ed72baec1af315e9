"""Arithmetic of the running statistics A and B (onmf_config.accumulate)
through the C ABI: FP64 (default), FP32, and compensated FP32 (a float pair
per entry).

  - every mode against the FP64 oracle on the small online workload
    (F=129, K=8, beta=50, 5 inner iterations, 40 minibatches), element-wise
    (helpers.parity): FP32 path within 1e-5 on W, A, B, H and the loss,
    mixed path within test_gpu_online.MIXED_TOL;
  - on a long stream (4,000 minibatches) the compensated pair stays with
    FP64 to float rounding of W, while plain FP32 sums drift further;
  - onmf_get_stats / onmf_set_state convert the float pairs to doubles and
    back, and a run resumed from them continues the uninterrupted run;
  - mixed path at the bench's shape (F=513, K=100, beta=1000): over four
    minibatches the compensated pairs equal the FP64 sums to 1e-13 relative
    per entry, with W bit-identical (the pairs carry about 48 bits).
"""
import numpy as np
import pytest

import paper_1106_4198_gb300 as onmf
from helpers import cuda, problem, relerr
from test_gpu_online import MIXED_TOL, compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
MODES = [onmf.ONMF_ACC_FP64, onmf.ONMF_ACC_FP32, onmf.ONMF_ACC_FP32_COMP]


@pytest.mark.parametrize("precision", [onmf.ONMF_FP32, onmf.ONMF_MIXED])
@pytest.mark.parametrize("acc", MODES)
def test_modes_match_oracle(acc, precision):
    F, K, N, beta, n_in = 129, 8, 2000, 50, 5
    V, W0 = problem(F, K, N, seed=3)
    g = run_gpu(V, W0, beta=beta, n_inner=n_in, precision=precision, accumulate=acc)
    o = run_oracle(V, W0, beta, n_in)
    tol = 1e-5 if precision == onmf.ONMF_FP32 else MIXED_TOL
    compare(g, o, tol, label="%s precision %d" % (onmf.ACC_NAMES[acc], precision))


def long_run(V, W0, acc, beta):
    m = onmf.OnlineISNMF(V.shape[1], W0.shape[0], W0, beta=beta, n_inner=3,
                         precision=onmf.ONMF_FP32, accumulate=acc)
    m.push(cuda(V))
    m.sync()
    W = m.W()
    A, B, t, ls = m.stats()
    m.close()
    return dict(W=W, A=A, B=B, t=t, loss=ls)


def test_long_stream_compensated_stays_with_fp64():
    F, K, N, beta = 65, 8, 200_000, 50
    V, W0 = problem(F, K, N, seed=11)
    r = {acc: long_run(V, W0, acc, beta) for acc in MODES}
    ref = r[onmf.ONMF_ACC_FP64]
    d = {onmf.ACC_NAMES[a]: {k: relerr(r[a][k], ref[k]) for k in ("W", "A", "B")}
         for a in MODES[1:]}
    print("4,000 minibatches, relative to FP64 sums:", d)
    assert all(x["t"] == N for x in r.values())
    comp, plain = d["fp32_compensated"], d["fp32"]
    # the pair carries ~2^-48 per step; what is left is float rounding of W'
    # fed back through the later minibatches
    assert comp["W"] <= 1e-5 and comp["A"] <= 1e-5 and comp["B"] <= 1e-5
    assert np.isfinite(plain["W"]) and plain["W"] <= 1e-2


@pytest.mark.parametrize("acc", [onmf.ONMF_ACC_FP32, onmf.ONMF_ACC_FP32_COMP])
def test_checkpoint_round_trip(acc):
    F, K, N, beta = 129, 8, 1200, 50
    V, W0 = problem(F, K, N, seed=13)
    Vd = cuda(V)
    full = onmf.OnlineISNMF(F, K, W0, beta=beta, n_inner=4, accumulate=acc)
    full.push(Vd)
    full.sync()
    Wf = full.W()
    full.close()
    a = onmf.OnlineISNMF(F, K, W0, beta=beta, n_inner=4, accumulate=acc)
    a.push(Vd[:600])
    a.sync()
    W, A, B, t, ls = a.W(), *a.stats()
    a.close()
    assert t == 600 and np.all(A > 0) and np.all(B > 0)
    b = onmf.OnlineISNMF(F, K, W0, beta=beta, n_inner=4, accumulate=acc)
    b.set_state(W, A, B, t, ls)
    A2, B2, t2, _ = b.stats()
    # a float pair holds a double to ~2^-48 (plain FP32: the float itself)
    lim = 2.0 ** -46 if acc == onmf.ONMF_ACC_FP32_COMP else 2.0 ** -23
    assert relerr(A2, A) <= lim and relerr(B2, B) <= lim and t2 == t
    b.push(Vd[600:])
    b.sync()
    e = relerr(b.W(), Wf)
    b.close()
    print(onmf.ACC_NAMES[acc], "resumed vs uninterrupted W: %.2e" % e)
    assert e <= 1e-5


@pytest.mark.parametrize("acc", [onmf.ONMF_ACC_FP32, onmf.ONMF_ACC_FP32_COMP])
@pytest.mark.parametrize("rho_on_new", [0, 1])
def test_forgetting_factor_in_every_mode(acc, rho_on_new):
    """rho = r^(beta'/n_ref) != 1 scales the past (or the new data) inside
    the float-pair arithmetic too."""
    F, K, N, beta = 129, 8, 1000, 50
    V, W0 = problem(F, K, N, seed=17)
    kw = dict(r=0.7, n_ref=N, rho_on_new=rho_on_new)
    g = run_gpu(V, W0, beta=beta, n_inner=3, accumulate=acc, **kw)
    o = run_oracle(V, W0, beta, 3, **kw)
    compare(g, o, 1e-5, label="forgetting factor %s rho_on_new=%d" % (onmf.ACC_NAMES[acc],
                                                                    rho_on_new))


def test_compensated_pairs_track_fp64_sums_mixed():
    F, K = 513, 100
    V, W0 = problem(F, K, 4000, seed=5)
    res = {}
    for acc in (onmf.ONMF_ACC_FP64, onmf.ONMF_ACC_FP32_COMP):
        m = onmf.OnlineISNMF(F, K, W0, beta=1000, n_inner=10, precision=onmf.ONMF_MIXED,
                             hsolve=onmf.ONMF_HSOLVE_MMA, accumulate=acc)
        m.push(cuda(V))
        m.sync()
        A, B, t, _ = m.stats()
        res[acc] = (m.W(), A, B)
        m.close()
    (W64, A64, B64), (Wc, Ac, Bc) = res[onmf.ONMF_ACC_FP64], res[onmf.ONMF_ACC_FP32_COMP]
    ea = float(np.max(np.abs(Ac - A64) / np.abs(A64)))
    eb = float(np.max(np.abs(Bc - B64) / np.abs(B64)))
    print("compensated vs FP64 after 4 minibatches: A %.2e B %.2e" % (ea, eb))
    assert np.array_equal(Wc, W64)
    assert ea <= 1e-13 and eb <= 1e-13
