"""Selecting the mixed-precision h-solve kernel (onmf_config.hsolve) and the
autotuner (onmf_autotune), through the C ABI.

  - a kernel chosen in the config gives the same bits as the same kernel
    chosen through the environment;
  - choices the shape does not allow are rejected;
  - the autotuner times every allowed schedule (kernel, and with the mma
    kernel the frame ranges of the statistics), returns the fastest, writes
    its cache and answers the next call from it; at K = 256 only the cluster
    kernel fits;
  - every statistics schedule gives the oracle's results within the
    one-minibatch bounds, and the same bits run to run."""
import json

import numpy as np
import pytest

import paper_1106_4198_gb300 as onmf
from helpers import problem
from test_gpu_online import MIXED_TOL, compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
MIXED = onmf.ONMF_MIXED


@pytest.mark.parametrize("hsolve", [onmf.ONMF_HSOLVE_MMA, onmf.ONMF_HSOLVE_TC,
                                    onmf.ONMF_HSOLVE_CLUSTER])
def test_config_choice_equals_environment_choice(hsolve, monkeypatch):
    F, K, beta = 513, 100, 300
    V, W0 = problem(F, K, 700, seed=71)
    monkeypatch.delenv("ONMF_HSOLVE", raising=False)
    a = run_gpu(V, W0, beta=beta, n_inner=4, precision=MIXED, hsolve=hsolve)
    monkeypatch.setenv("ONMF_HSOLVE", onmf.HSOLVE_NAMES[hsolve])
    b = run_gpu(V, W0, beta=beta, n_inner=4, precision=MIXED)
    for k in ("W", "A", "B", "H"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("F,K,hsolve", [(129, 200, onmf.ONMF_HSOLVE_MMA),
                                        (129, 200, onmf.ONMF_HSOLVE_TC),
                                        (60, 8, onmf.ONMF_HSOLVE_TC)])
def test_choices_the_shape_does_not_allow_are_rejected(F, K, hsolve):
    W0 = np.full((K, F), 1.0 / F, dtype=np.float32)
    with pytest.raises(onmf.OnmfError) as e:
        onmf.OnlineISNMF(F, K, W0, precision=MIXED, hsolve=hsolve)
    assert e.value.status == 1  # ONMF_EINVAL


def test_autotune_picks_the_fastest_and_caches(tmp_path):
    cache = str(tmp_path / "tune.jsonl")
    cfg = onmf.onmf_config_default(513, 100, precision=MIXED, beta=1000, n_inner=10)
    h, sr, times, ranges, hit = onmf.onmf_autotune(cfg, cache)
    print("autotune F=513 K=100 beta=1000:", onmf.HSOLVE_NAMES[h], "stats_ranges", sr, times,
          ranges)
    assert not hit and set(times) == {"mma", "tc", "cluster"}
    assert set(ranges) == set(onmf.STATS_RANGE_CANDIDATES)
    assert onmf.HSOLVE_NAMES[h] == min(times, key=times.get)
    assert times["mma"] == min(ranges.values())
    if h == onmf.ONMF_HSOLVE_MMA:
        assert ranges[sr] == min(ranges.values())
    line = json.loads(open(cache).read().splitlines()[-1])
    assert (line["F"], line["K"], line["beta"], line["n_inner"], line["hsolve"],
            line["stats_ranges"]) == (513, 100, 1000, 10, h, sr)
    assert line["tile_frames"] == {1: 8, 2: 16, 3: 32}[h]
    h2, sr2, _, _, hit2 = onmf.onmf_autotune(cfg, cache)
    assert hit2 and h2 == h and sr2 == sr
    # a state built with the tuned choice runs
    V, W0 = problem(513, 100, 2000, seed=72)
    g = run_gpu(V, W0, beta=1000, n_inner=10, precision=MIXED, hsolve=h, stats_ranges=sr)
    assert g["t"] == 2000 and np.all(np.isfinite(g["W"]))


def test_autotune_k256_has_only_the_cluster_kernel():
    cfg = onmf.onmf_config_default(513, 256, precision=MIXED, beta=512, n_inner=5)
    h, sr, times, ranges, hit = onmf.onmf_autotune(cfg)
    assert h == onmf.ONMF_HSOLVE_CLUSTER and set(times) == {"cluster"} and not hit
    assert ranges == {} and sr == 0


@pytest.mark.parametrize("ranges", [1, 2, 5, 16, 256])
def test_statistics_schedules_match_the_oracle(ranges):
    """The frame ranges of the statistics change only the order of the
    FP32 sums over frames: each schedule stays within the one-minibatch
    bounds of the oracle (a ragged stream: full minibatches and a flushed
    partial one), and a schedule gives the same bits twice."""
    F, K, beta, n_in = 513, 100, 1000, 5
    V, W0 = problem(F, K, 2333, seed=73)
    a = run_gpu(V, W0, beta=beta, n_inner=n_in, precision=MIXED,
                hsolve=onmf.ONMF_HSOLVE_MMA, stats_ranges=ranges)
    b = run_gpu(V, W0, beta=beta, n_inner=n_in, precision=MIXED,
                hsolve=onmf.ONMF_HSOLVE_MMA, stats_ranges=ranges)
    for k in ("W", "A", "B", "H"):
        assert np.array_equal(a[k], b[k]), k
    o = run_oracle(V, W0, beta, n_in)
    compare(a, o, MIXED_TOL, label="stats_ranges=%d" % ranges)
