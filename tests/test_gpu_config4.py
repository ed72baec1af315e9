"""The mixed-precision settings of the K x beta grid over a whole pass of the
objective-vs-time workload: F = 513, N = 112,500 frames of the gamma model
(drawn with a 50-atom W*), dictionaries of K in {64, 100, 256} atoms,
minibatches beta in {512, 2048}, 10 inner iterations, the h-solve kernel the
autotuner picks. Every setting against the FP64 oracle over the same pass:
the error of W, A, B and of the running objective is printed and held to the
mixed-path bounds (1e-2 on W, A, B; 1e-3 on the objective)."""
import numpy as np
import pytest

import paper_1106_4198_gb300 as onmf
import synth
from helpers import relerr
from test_gpu_online import run_gpu, run_oracle

pytestmark = pytest.mark.gpu
F, N, N_IN = 513, 112_500, 10


@pytest.fixture(scope="module")
def frames():
    return synth.spectrogram(F, 50, N, seed=synth.DATA_SEED + 2)


@pytest.mark.parametrize("beta", [512, 2048])
@pytest.mark.parametrize("K", [64, 100, 256])
def test_setting_full_pass(K, beta, frames, tmp_path):
    cfg = onmf.onmf_config_default(F, K, precision=onmf.ONMF_MIXED, beta=beta, n_inner=N_IN)
    h, times, _ = onmf.onmf_autotune(cfg, str(tmp_path / "tune.jsonl"))
    W0 = synth.init_dictionary(F, K)
    g = run_gpu(frames, W0, beta=beta, n_inner=N_IN, precision=onmf.ONMF_MIXED, hsolve=h,
                want_H=False)
    o = run_oracle(frames, W0, beta, N_IN)
    e = dict(W=relerr(g["W"], o["W"]), A=relerr(g["A"], o["A"]), B=relerr(g["B"], o["B"]),
             objective=abs(g["loss_sum"] - o["loss_sum"]) / o["loss_sum"])
    print("K=%d beta=%d h-solve %s (%s): objective %.6f" % (
        K, beta, onmf.HSOLVE_NAMES[h], {k: round(v, 1) for k, v in times.items()},
        o["loss_sum"] / N), {k: "%.2e" % v for k, v in e.items()})
    assert g["t"] == N
    assert e["objective"] <= 1e-3
    for k in ("W", "A", "B"):
        assert e[k] <= 1e-2, (k, e)
