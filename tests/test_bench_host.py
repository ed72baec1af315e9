"""Host logic of bench.py without a GPU: the multi-rank helpers on gloo
(world size 2, CPU), the reference arm's JSON line and rank gating, and the
serving arrival schedule."""
import json
import os
import socket

import numpy as np
import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    r, w, local = bench.dist_env()
    dist = bench.init_dist(w, "gloo")
    bench.barrier(dist)
    res = {
        "env": [r, w, local],
        "max": bench.max_over_ranks(dist, 10.0 * (rank + 1)),
        "sum": bench.sum_over_ranks(dist, 1000.0 + rank),
    }

    class A:
        steps, warmup = 1, 0
    # the reference arm runs on rank 0 only; the other ranks return no line
    res["ref_none"] = bench.run_reference(A) is None if rank != 0 else None
    bench.barrier(dist)
    dist.destroy_process_group()
    with open(os.path.join(outdir, "rank%d.json" % rank), "w") as f:
        json.dump(res, f)


def test_two_rank_helpers_on_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2,
                       join=True, start_method="spawn")
    r0 = json.load(open(tmp_path / "rank0.json"))
    r1 = json.load(open(tmp_path / "rank1.json"))
    assert r0["env"] == [0, 2, 0] and r1["env"] == [1, 2, 1]
    # time = max over ranks, units = sum over ranks, identical on every rank
    assert r0["max"] == r1["max"] == 20.0
    assert r0["sum"] == r1["sum"] == 2001.0
    assert r1["ref_none"] is True


def test_single_rank_helpers_are_identity(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.init_dist(1, "gloo") is None
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.sum_over_ranks(None, 7.0) == 7.0


def test_reference_line_keys(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)

    class A:
        steps, warmup = 1, 0
    out = bench.run_reference(A)
    assert out["impl"] == "reference" and out["metric"] == bench.METRIC
    assert out["unit"] == "frames/s" and out["higher_is_better"] is True
    assert out["value"] > 0 and out["cpu_baseline"]["kind"] == "oracle"
    assert out["cpu_baseline"]["value"] == out["value"]
    assert out["e2e"] == {"value": out["value"], "unit": "frames/s",
                          "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    json.dumps(out)


def test_serving_schedule_shape():
    rng = np.random.default_rng(4321)
    Ks, events = bench.serving_schedule(64, 30.0, rng)
    assert len(Ks) == 64 and set(Ks) <= set(bench.SERVE_KS)
    t = [e[0] for e in events]
    assert t == sorted(t) and 0 <= t[0] and t[-1] < 30.0
    sizes = np.array([e[2] for e in events])
    assert sizes.min() >= 1 and sizes.max() <= 512
    # full-length chunks are log-uniform over [8, 512]: median near sqrt(8*512)
    assert 30 <= np.median(sizes) <= 100
    # each stream delivers frames at about 4x real time while it is active
    # (Poisson chunk arrivals; short streams end inside the window)
    rates = []
    for i in range(64):
        ev = [e for e in events if e[1] == i]
        if len(ev) >= 20:
            rates.append(sum(e[2] for e in ev[1:]) / (ev[-1][0] - ev[0][0]))
    target = bench.SPEEDUP / bench.HOP_S
    assert len(rates) >= 10
    assert 0.8 * target <= np.median(rates) <= 1.25 * target


def test_accumulator_choice_rule():
    """The fastest arithmetic of A, B whose drift against the FP64 sums is
    within the bounds; FP64 whenever nothing else qualifies."""
    def d(fp32_w, fp32_ms, comp_w, comp_ms, fp64_ms=45.8):
        return {"fp64": {"ms_per_1e6_frames": fp64_ms},
                "fp32": {"ms_per_1e6_frames": fp32_ms, "W_rel": fp32_w, "A_rel": fp32_w,
                         "B_rel": fp32_w},
                "fp32_compensated": {"ms_per_1e6_frames": comp_ms, "W_rel": comp_w,
                                     "A_rel": comp_w * 1e-6, "B_rel": comp_w * 1e-6}}
    # plain FP32 is fastest but drifts; the compensated pair does not
    assert bench.choose_accumulate(d(9e-6, 45.0, 0.0, 45.2)) == "fp32_compensated"
    # nothing qualifying is faster than FP64
    assert bench.choose_accumulate(d(9e-6, 45.0, 0.0, 46.0)) == "fp64"
    # every candidate drifts
    assert bench.choose_accumulate(d(9e-6, 45.0, 5e-6, 45.1)) == "fp64"
    # a plain FP32 run within the bounds is taken when it is the fastest
    assert bench.choose_accumulate(d(1e-12, 44.0, 0.0, 45.2)) == "fp32"


def test_unfused_comparison_leg_computes_algorithm_1():
    """The benchmark's unfused FP32 leg (PyTorch ops) run in FP64 on the CPU
    gives the oracle's W, A, B over a few minibatches (to rounding)."""
    import torch
    import oracle
    import synth
    F, K, beta, n_in = 33, 4, 8, 3
    V = synth.spectrogram(F, K, 3 * beta, seed=3)
    W0 = synth.init_dictionary(F, K)
    Vt = torch.as_tensor(V, dtype=torch.float64)
    W = torch.as_tensor(W0, dtype=torch.float64).t().contiguous()
    A, B = torch.zeros_like(W), torch.zeros_like(W)
    for j in range(3):
        W, A, B = bench.unfused_minibatch(Vt[j * beta:(j + 1) * beta], W, A, B, 1e-12, n_in)
    o = oracle.online_pass(V, W0, beta=beta, n_in=n_in)
    for x, ref in ((W, o["W"]), (A, o["A"]), (B, o["B"])):
        assert np.allclose(x.t().numpy(), ref, rtol=1e-12, atol=0)
