"""Parity at the benchmark's sizes and in its launch configuration: F = 513,
K = 100, beta = 1000, 10 inner iterations, mixed precision with the mma
h-solve and compensated FP32 sums (the bench's measured choices), 10^6
frames drawn on the device by the bench's generator and pushed in ONE call
(one persistent launch over 1,000 minibatches).

The oracle cannot redo 10^6 frames in a test, so:
  - properties that hold at any size, over the whole launch: the same
    frames pushed in pieces (with checkpoints read in between) give the
    single launch's W, A, B, H and running loss bit for bit; W >= 0 with
    unit column sums; A, B, H >= 0 and finite; one kernel launch;
  - sampled minibatches recomputed by the FP64 oracle from the GPU's own
    state before them (minibatch 500 and the last one): W, A, B after the
    step, the h of every frame of the minibatch and the loss increment,
    element-wise within FULL_TOL (rows of W, A, B including the last).
"""
import numpy as np
import pytest

import oracle
import paper_1106_4198_gb300 as onmf
import synth
from helpers import parity
from test_gpu_online import MIXED_TOL

# W, A, B after one step from a state of 500+ minibatches move little, so
# their bounds are about three times the measured (W 1.0e-6, A 3.5e-6,
# B 2.0e-6 per entry); H as for one minibatch.
FULL_TOL = dict(W=3e-6, A=1.1e-5, B=6e-6, H=MIXED_TOL["H"], loss=MIXED_TOL["loss"])

pytestmark = pytest.mark.gpu
F, K, BETA, N_IN, N = 513, 100, 1000, 10, 1_000_000
CFG = dict(beta=BETA, n_inner=N_IN, precision=onmf.ONMF_MIXED, hsolve=onmf.ONMF_HSOLVE_MMA,
           accumulate=onmf.ONMF_ACC_FP32_COMP)


@pytest.fixture(scope="module")
def frames():
    import torch
    Wstar = torch.as_tensor(synth.dictionary(F, K, synth.DATA_SEED), dtype=torch.float32,
                            device="cuda")
    V = synth.device_frames(F, K, N, seed=synth.DATA_SEED, chunk=0, Wstar=Wstar)
    torch.cuda.synchronize()
    return V


def snapshot(m):
    m.sync()
    A, B, t, ls = m.stats()
    return dict(W=m.W(), A=A, B=B, t=t, loss=ls)


@pytest.fixture(scope="module")
def runs(frames):
    import torch
    W0 = synth.init_dictionary(F, K)
    # the bench's launch: every frame in one push
    H1 = torch.empty((N, K), device="cuda")
    m = onmf.OnlineISNMF(F, K, W0, **CFG)
    l0 = onmf.onmf_kernel_launches()
    m.push(frames, H1)
    one = snapshot(m)
    one["launches"] = onmf.onmf_kernel_launches() - l0
    m.close()
    # the same frames in pieces, state read before minibatches 500 and 1000
    cuts = [0, 499 * BETA, 500 * BETA, 999 * BETA, N]
    H2 = torch.empty((N, K), device="cuda")
    m = onmf.OnlineISNMF(F, K, W0, **CFG)
    snaps = [snapshot(m)]
    for a, b in zip(cuts[:-1], cuts[1:]):
        m.push(frames[a:b], H2[a:b])
        snaps.append(snapshot(m))
    m.close()
    return one, H1, snaps, H2, cuts


def test_one_launch_and_its_invariants(runs):
    one, H1, snaps, H2, _ = runs
    assert one["t"] == N
    assert one["launches"] == 1  # one persistent launch for the 1,000 minibatches
    W = one["W"]
    assert np.all(W >= 0) and np.all(np.isfinite(W))
    assert np.max(np.abs(W.sum(axis=1) - 1.0)) <= 1e-5  # L1 rescale of every column
    for X in (one["A"], one["B"]):
        assert np.all(X >= 0) and np.all(np.isfinite(X))
    h = H1.cpu().numpy()
    assert np.all(h >= 0) and np.all(np.isfinite(h))


def test_pieces_equal_the_single_launch_bitwise(runs):
    one, H1, snaps, H2, _ = runs
    last = snaps[-1]
    for k in ("W", "A", "B"):
        assert np.array_equal(last[k], one[k]), k
    assert last["loss"] == one["loss"] and last["t"] == one["t"]
    assert bool((H1 == H2).all())


@pytest.mark.parametrize("piece", [1, 3])  # minibatch 500 and minibatch 1000
def test_sampled_minibatch_against_oracle(runs, frames, piece):
    one, H1, snaps, H2, cuts = runs
    before, after = snaps[piece], snaps[piece + 1]
    a, b = cuts[piece], cuts[piece + 1]
    assert b - a == BETA and before["t"] == a
    V = frames[a:b].cpu().numpy()
    oracle.set_threads(16)
    o = oracle.online_pass(V, before["W"], before["A"], before["B"], beta=BETA, n_in=N_IN)
    oracle.set_threads(1)
    parity("minibatch %d of 1000 at full size" % (b // BETA),
           dict(W=(after["W"], o["W"]), A=(after["A"], o["A"]), B=(after["B"], o["B"]),
                H=(H1[a:b].cpu().numpy(), o["H"]),
                loss=(after["loss"] - before["loss"], o["loss_sum"])), FULL_TOL)
