"""Guard bands around every caller-owned buffer (the stand-in for a memory
sanitizer, which is closed on this machine): outputs live inside larger
allocations whose margins and padding columns hold a canary value, inputs
carry NaN in their padding columns and must come back unchanged. After each
call through the C ABI the margins must still hold the canary bit for bit, so
a write outside an output's logical extent fails the test; a read of an
input's padding would meet NaN, which the kernels' input check reports as
an error. Shapes are odd and ragged (F = 1, 17, 129, 513; K = 1, 3, 100, 200;
beta = 1, 7, 50, 1000; partial minibatches; a flush) on every h-solve kernel
that takes them, with device and host input."""
import numpy as np
import pytest

import paper_1106_4198_gb300 as onmf
from helpers import problem

pytestmark = pytest.mark.gpu
CANARY = -12345.678
G = 3  # guard rows before and after
PADC = 5  # guard columns


def guarded(n, cols, device=True, fill=CANARY):
    """(buffer, view): the view is (n, cols) inside a buffer with G guard rows
    before and after and PADC guard columns (row stride cols + PADC)."""
    import torch
    buf = torch.full((n + 2 * G, cols + PADC), fill, dtype=torch.float32)
    if device:
        buf = buf.cuda()
    return buf, buf[G:G + n, :cols]


def margins_intact(buf, n, cols):
    import torch
    b = buf.cpu()
    inner = torch.zeros_like(b, dtype=torch.bool)
    inner[G:G + n, :cols] = True
    return bool((b[~inner] == CANARY).all())


def padded_input(V, device=True):
    """V (n, F) copied into a buffer whose padding columns and margin rows are
    NaN; returns (buffer, view)."""
    import torch
    n, F = V.shape
    buf, view = guarded(n, F, device=device, fill=float("nan"))
    view.copy_(torch.as_tensor(V))
    return buf, view


SHAPES = [(1, 1, 1, 5), (17, 3, 7, 40), (129, 100, 50, 333), (513, 100, 1000, 2100),
          (65, 200, 32, 75)]
KERNELS = [(onmf.ONMF_FP32, 0), (onmf.ONMF_MIXED, onmf.ONMF_HSOLVE_MMA),
           (onmf.ONMF_MIXED, onmf.ONMF_HSOLVE_TC), (onmf.ONMF_MIXED, onmf.ONMF_HSOLVE_CLUSTER)]


def make_state(F, K, beta, precision, hsolve, W0):
    try:
        return onmf.OnlineISNMF(F, K, W0, beta=beta, n_inner=3, precision=precision,
                                hsolve=hsolve)
    except onmf.OnmfError as e:
        if e.status == 1:  # this kernel does not take the shape
            pytest.skip(str(e))
        raise


@pytest.mark.parametrize("precision,hsolve", KERNELS)
@pytest.mark.parametrize("F,K,beta,n", SHAPES)
@pytest.mark.parametrize("device_input", [True, False])
def test_online_push_get_w_project(F, K, beta, n, precision, hsolve, device_input):
    import torch
    V, W0 = problem(F, K, n, seed=F + K + beta)
    m = make_state(F, K, beta, precision, hsolve, W0)
    vbuf, v = padded_input(V, device=device_input)
    vbuf0 = vbuf.clone()
    hbuf, h = guarded(n, K)
    # ragged pushes, then a flush
    cuts = [0, n // 3, n // 3 + 1, n]
    for a, b in zip(cuts[:-1], cuts[1:]):
        if b > a:
            m.push(v[a:b] if device_input else v[a:b].numpy(), h[a:b])
    m.flush()
    m.sync()
    _, _, t, _ = m.stats()
    assert t == n
    assert margins_intact(hbuf, n, K), "h output written outside its extent"
    assert torch.equal(vbuf.isnan(), vbuf0.isnan()) and torch.equal(
        torch.nan_to_num(vbuf), torch.nan_to_num(vbuf0)), "input frames modified"
    # W into a guarded (K, F) buffer (contiguous rows are required there)
    import torch as th
    wbuf = th.full((K * F + 2 * 64,), CANARY, device="cuda")
    onmf.onmf_get_W(m.state, wbuf[64:64 + K * F].view(K, F))
    wb = wbuf.cpu()
    assert bool((wb[:64] == CANARY).all() and (wb[64 + K * F:] == CANARY).all())
    # projection with W fixed into another guarded output
    pbuf, p = guarded(n, K)
    m.project(v if device_input else v.numpy(), p, n_inner=2)
    m.sync()
    assert margins_intact(pbuf, n, K), "projection written outside its extent"
    m.close()


@pytest.mark.parametrize("precision,hsolve", KERNELS[:2])
def test_warm_restart_buffers(precision, hsolve):
    import torch
    F, K, beta, n = 129, 8, 16, 70
    V, W0 = problem(F, K, n, seed=7)
    m = make_state(F, K, beta, precision, hsolve, W0)
    vbuf, v = padded_input(V)
    hbuf, h = guarded(n, K)
    h.fill_(1.0)
    order = torch.randperm(n, generator=torch.Generator().manual_seed(3)).cuda()
    m.push_warm(v, h, order)
    m.flush()
    m.sync()
    m.close()
    assert margins_intact(hbuf, n, K)
    assert bool(torch.isfinite(h).all())


@pytest.mark.parametrize("precision", [onmf.ONMF_FP32, onmf.ONMF_MIXED])
def test_batch_step_buffers(precision):
    import torch
    F, K, n = 129, 8, 301
    V, W0 = problem(F, K, n, seed=9)
    vbuf, v = padded_input(V)
    wb = torch.full((K * F + 128,), CANARY, device="cuda")
    hb = torch.full((n * K + 128,), CANARY, device="cuda")
    W = wb[64:64 + K * F].view(K, F)
    H = hb[64:64 + n * K].view(n, K)
    W.copy_(torch.as_tensor(W0))
    onmf.nmf_batch_init_H(v, W, H)
    onmf.nmf_batch_step(v, W, H, n_iter=3, precision=precision)
    torch.cuda.synchronize()
    for b, m in ((wb, K * F), (hb, n * K)):
        c = b.cpu()
        assert bool((c[:64] == CANARY).all() and (c[64 + m:] == CANARY).all())


def test_serving_host_buffers():
    F = 129
    srv = onmf.onmf_server_create(F, max_chunk=512, max_batch=8, slots=2,
                                  precision=onmf.ONMF_MIXED)
    try:
        outs = []
        for i, (K, n) in enumerate([(16, 9), (64, 100), (128, 33)]):
            V, W0 = problem(F, K, n, seed=20 + i)
            sid = onmf.onmf_server_open_stream(
                srv, onmf.onmf_config_default(F, K, precision=onmf.ONMF_MIXED, n_inner=3), W0)
            buf = np.full((n + 2 * G, K), CANARY, dtype=np.float32)
            onmf.onmf_server_submit(srv, sid, V, tag=i, H_out=buf[G:G + n])
            outs.append((buf, n))
        got = 0
        while got < len(outs):
            for cp in onmf.onmf_server_poll(srv, 16, wait_ms=2000):
                assert cp.status == 0
                got += 1
    finally:
        onmf.onmf_server_destroy(srv)
    for buf, n in outs:
        assert np.all(buf[:G] == CANARY) and np.all(buf[G + n:] == CANARY)
        assert np.all(np.isfinite(buf[G:G + n])) and np.all(buf[G:G + n] != CANARY)
