"""Serving: many streams, each its own run of Algorithm 1, fed chunk by chunk
through onmf_server_* (C ABI). Every chunk is one minibatch of its stream.

Checked here:
  - one stream served chunk by chunk equals the single-state path
    (onmf_push_frames + onmf_flush per chunk), bit for bit;
  - a stream's results alone equal its results in a mix of streams with
    other dictionary sizes and chunk lengths, bit for bit;
  - parity with the FP64 oracle run chunk by chunk, W element-wise and by
    frequency row (FP32 <= 1e-5; mixed <= 4e-3, three times the measured
    1.2e-3), every chunk's loss within 1e-5 / 1e-3;
  - admission by the memory budget: streams that do not fit wait and run
    once others close;
  - batches launched as captured CUDA graphs (the default) and as direct
    kernel launches give the same bits.
"""
import numpy as np
import pytest

import oracle
import paper_1106_4198_gb300 as onmf
from helpers import cuda, parity, problem

pytestmark = pytest.mark.gpu


def chunks_of(n_total, rng, lo=8, hi=64):
    sizes = []
    while sum(sizes) < n_total:
        sizes.append(int(min(rng.integers(lo, hi + 1), n_total - sum(sizes))))
    return sizes


def serve(streams, precision, budget=1 << 30, max_batch=64, close_early=None,
          launch=onmf.ONMF_SERVE_GRAPH):
    """streams: list of (V (N,F), W0 (K,F), sizes, cfg kwargs). Submits every
    chunk of every stream interleaved; returns per-stream (W, chunk losses)."""
    F = streams[0][0].shape[1]
    srv = onmf.onmf_server_create(F, max_chunk=512, max_batch=max_batch, slots=2,
                                  budget_bytes=budget, precision=precision, launch=launch)
    try:
        ids = []
        for V, W0, sizes, kw in streams:
            K = W0.shape[0]
            cfg = onmf.onmf_config_default(F, K, precision=precision, **kw)
            ids.append(onmf.onmf_server_open_stream(srv, cfg, W0))
        offs = [0] * len(streams)
        k = [0] * len(streams)
        pending = sum(len(s[2]) for s in streams)
        order = []
        while len(order) < pending:
            for i, (V, W0, sizes, kw) in enumerate(streams):
                if k[i] < len(sizes):
                    order.append((i, k[i]))
                    k[i] += 1
        for i, c in order:
            V, W0, sizes, kw = streams[i]
            a = sum(sizes[:c])
            onmf.onmf_server_submit(srv, ids[i], V[a:a + sizes[c]], tag=c)
        losses = [dict() for _ in streams]
        got = 0
        pos = {sid: i for i, sid in enumerate(ids)}
        while got < pending:
            for cp in onmf.onmf_server_poll(srv, 256, wait_ms=2000):
                assert cp.status == 0
                losses[pos[cp.stream_id]][cp.tag] = cp.loss
                got += 1
        out = []
        for i, (V, W0, sizes, kw) in enumerate(streams):
            W = onmf.onmf_server_get_W(srv, ids[i], W0.shape[0], F)
            out.append((W, [losses[i][c] for c in range(len(sizes))]))
        stats = onmf.onmf_server_get_stats(srv)
    finally:
        onmf.onmf_server_destroy(srv)
    return out, stats


def single_state(V, W0, sizes, precision, **kw):
    K, F = W0.shape
    m = onmf.OnlineISNMF(F, K, W0, beta=512, precision=precision, **kw)
    Vd = cuda(V)
    losses = []
    prev = 0.0
    a = 0
    for n in sizes:
        m.push(Vd[a:a + n])
        m.flush()
        _, _, _, ls = m.stats()
        losses.append(ls - prev)
        prev = ls
        a += n
    W = m.W()
    m.close()
    return W, losses


@pytest.mark.parametrize("precision", [onmf.ONMF_FP32, onmf.ONMF_MIXED])
def test_served_stream_equals_single_state_path(precision):
    F, K = 129, 16
    V, W0 = problem(F, K, 400)
    sizes = chunks_of(400, np.random.default_rng(1))
    (W, losses), = serve([(V, W0, sizes, dict(n_inner=5))], precision)[0]
    Ws, ls = single_state(V, W0, sizes, precision, n_inner=5)
    assert np.array_equal(W, Ws)
    # per-chunk losses: served values are exact, single-state ones are
    # differences of the running sum (rounding of the subtraction)
    assert np.allclose(losses, ls, rtol=1e-9)


@pytest.mark.parametrize("precision", [onmf.ONMF_FP32, onmf.ONMF_MIXED])
def test_result_alone_equals_result_in_the_mix(precision):
    rng = np.random.default_rng(2)
    F = 129
    target_V, target_W0 = problem(F, 32, 600, seed=7)
    target_sizes = chunks_of(600, rng, 8, 128)
    target = (target_V, target_W0, target_sizes, dict(n_inner=6))
    alone, _ = serve([target], precision)
    others = []
    for i in range(23):
        K = int(rng.choice([16, 32, 64, 128]))
        N = int(rng.integers(100, 700))
        V, W0 = problem(F, K, N, seed=100 + i)
        others.append((V, W0, chunks_of(N, rng, 8, 256), dict(n_inner=6)))
    mixed, stats = serve(others[:11] + [target] + others[11:], precision, max_batch=32)
    W_alone, l_alone = alone[0]
    W_mix, l_mix = mixed[11]
    assert np.array_equal(W_alone, W_mix)
    assert l_alone == l_mix
    print("mix stats:", stats)
    assert stats["chunks"] == sum(len(s[2]) for s in others) + len(target_sizes)


@pytest.mark.parametrize("precision,tol_w,tol_l", [(onmf.ONMF_FP32, 1e-5, 1e-5),
                                                   (onmf.ONMF_MIXED, 4e-3, 1e-3)])
def test_served_streams_match_oracle(precision, tol_w, tol_l):
    rng = np.random.default_rng(3)
    F = 129
    streams = []
    for i, K in enumerate([16, 32, 64, 128]):
        V, W0 = problem(F, K, 300, seed=40 + i)
        streams.append((V, W0, chunks_of(300, rng, 8, 100), dict(n_inner=5, r=0.7, n_ref=300)))
    out, _ = serve(streams, precision)
    for (V, W0, sizes, kw), (W, losses) in zip(streams, out):
        Wo, Ao, Bo = W0.astype(np.float64), None, None
        lo = []
        a = 0
        for n in sizes:
            o = oracle.online_pass(V[a:a + n], Wo, Ao, Bo, beta=n, n_in=5, r=0.7, n_ref=300)
            Wo, Ao, Bo = o["W"], o["A"], o["B"]
            lo.append(o["loss_sum"])
            a += n
        el = np.max(np.abs(np.array(losses) - lo) / np.array(lo))
        print("K=%d: worst chunk loss rel err %.2e" % (W0.shape[0], el))
        assert el <= tol_l
        parity("served stream K=%d prec=%d" % (W0.shape[0], precision), dict(W=(W, Wo)), tol_w)


def test_one_launch_equals_launch_per_size_bitwise(monkeypatch):
    """The h-solve of a batch mixing dictionary sizes runs as one launch
    (the mma h-solve reads each chunk's size at run time) or, with
    ONMF_SERVE_FORK=1, as one launch per size of kernels specialized by
    size: the same operations in the same order, the same bits."""
    rng = np.random.default_rng(9)
    F = 129
    streams = []
    for i, K in enumerate([16, 48, 100, 128, 24]):
        V, W0 = problem(F, K, 200, seed=70 + i)
        streams.append((V, W0, chunks_of(200, rng, 8, 120), dict(n_inner=4)))
    one, _ = serve(streams, onmf.ONMF_MIXED)
    monkeypatch.setenv("ONMF_SERVE_FORK", "1")
    fork, _ = serve(streams, onmf.ONMF_MIXED)
    for (Wa, la), (Wb, lb) in zip(one, fork):
        assert np.array_equal(Wa, Wb)
        assert la == lb


def test_admission_by_budget():
    F, K = 129, 64
    srv = onmf.onmf_server_create(F, max_chunk=128, max_batch=16, slots=2,
                                  budget_bytes=500_000, precision=onmf.ONMF_MIXED)
    try:
        ids = []
        data = []
        for i in range(4):
            V, W0 = problem(F, K, 64, seed=60 + i)
            cfg = onmf.onmf_config_default(F, K, precision=onmf.ONMF_MIXED, n_inner=3)
            ids.append(onmf.onmf_server_open_stream(srv, cfg, W0))
            data.append(V)
        st = onmf.onmf_server_get_stats(srv)
        assert st["streams_admitted"] < 4 and st["streams_pending"] > 0
        for sid, V in zip(ids, data):
            onmf.onmf_server_submit(srv, sid, V, tag=sid)
        done = set()
        # the admitted streams finish; closing them lets the waiting ones in
        for _ in range(200):
            for cp in onmf.onmf_server_poll(srv, 16, wait_ms=50):
                assert cp.status == 0
                done.add(cp.stream_id)
                onmf.onmf_server_close_stream(srv, cp.stream_id)
            if len(done) == 4:
                break
        assert done == set(ids)
        st = onmf.onmf_server_get_stats(srv)
        assert st["streams_admitted"] == 4 and st["streams_pending"] == 0
    finally:
        onmf.onmf_server_destroy(srv)


@pytest.mark.parametrize("precision", [onmf.ONMF_FP32, onmf.ONMF_MIXED])
def test_graph_launch_equals_direct_launch(precision):
    """Every K of the serving mix, ragged chunks, small batches (so that the
    same set of dictionary sizes recurs with other layouts and each slot
    replays its graphs many times)."""
    rng = np.random.default_rng(5)
    F = 129
    streams = []
    for i, K in enumerate([16, 32, 64, 128, 16, 64]):
        N = int(rng.integers(150, 500))
        V, W0 = problem(F, K, N, seed=200 + i)
        streams.append((V, W0, chunks_of(N, rng, 8, 200), dict(n_inner=4)))
    g, sg = serve(streams, precision, max_batch=4, launch=onmf.ONMF_SERVE_GRAPH)
    d, sd = serve(streams, precision, max_batch=4, launch=onmf.ONMF_SERVE_DIRECT)
    print("graph:", sg, "direct:", sd)
    for (Wg, lg), (Wd, ld) in zip(g, d):
        assert np.array_equal(Wg, Wd)
        assert lg == ld
    assert sg["chunks"] == sd["chunks"] == sum(len(s[2]) for s in streams)


def test_submit_many_equals_submit_one_by_one():
    """One onmf_server_submit_many call per stream gives the bits of one
    onmf_server_submit call per chunk; H_out rows arrive for the chunks that
    ask for them."""
    rng = np.random.default_rng(9)
    F = 129
    streams = []
    for i, K in enumerate([16, 64, 32]):
        N = int(rng.integers(120, 300))
        V, W0 = problem(F, K, N, seed=300 + i)
        streams.append((V, W0, chunks_of(N, rng, 8, 100), dict(n_inner=3)))
    ref, _ = serve(streams, onmf.ONMF_MIXED)
    srv = onmf.onmf_server_create(F, max_chunk=512, max_batch=8, slots=2,
                                  precision=onmf.ONMF_MIXED)
    try:
        ids, total, Hs = [], 0, []
        for V, W0, sizes, kw in streams:
            cfg = onmf.onmf_config_default(F, W0.shape[0], precision=onmf.ONMF_MIXED, **kw)
            ids.append(onmf.onmf_server_open_stream(srv, cfg, W0))
        for (V, W0, sizes, kw), sid in zip(streams, ids):
            starts = np.cumsum([0] + sizes[:-1])
            Vs = [V[a:a + n] for a, n in zip(starts, sizes)]
            H = [np.zeros((n, W0.shape[0]), np.float32) if c % 2 == 0 else None
                 for c, n in enumerate(sizes)]
            Hs.append(H)
            assert onmf.onmf_server_submit_many(srv, [sid] * len(sizes), Vs,
                                                list(range(len(sizes))), H) == len(sizes)
            total += len(sizes)
        got = 0
        while got < total:
            for cp in onmf.onmf_server_poll(srv, 256, wait_ms=2000):
                assert cp.status == 0
                got += 1
        for i, ((V, W0, sizes, kw), sid) in enumerate(zip(streams, ids)):
            W = onmf.onmf_server_get_W(srv, sid, W0.shape[0], F)
            assert np.array_equal(W, ref[i][0])
            assert all(h is None or (np.all(np.isfinite(h)) and h.max() > 0) for h in Hs[i])
        with pytest.raises(onmf.OnmfError):  # unknown stream: refused
            onmf.onmf_server_submit_many(srv, [12345], [V[:8]], [0])
    finally:
        onmf.onmf_server_destroy(srv)
