"""The allocation-free projection (onmf_project_static), called through the
C ABI, against the regular projection (onmf_project) on the same inputs.

onmf_project_static serves callers that cannot allocate device memory: a
real-time audio callback, where cudaMalloc may stall on a device-wide
synchronization, and hosts that hand the library a fixed memory arena and
forbid allocations of its own. Its scratch is one static device array shared
by all calls, so the tests make calls in a row with different shapes and
precisions (a call must not see the leftovers of the one before).

Both entry points run the same tile kernels on the same derived images of W
(the same preparation kernel makes them), every frame tile's h and loss slot
depend only on that tile, and the loss slots are summed by the same
fixed-order kernel, so the two must agree bit for bit: H and the objective
are compared with exact equality.

The file is collected last (its name), so a run that stops at the first
failure has run every other test already. The first-call path (looking up
the array's device address on a device that has not used the entry point)
runs in a fresh subprocess, as it would in a new process of a caller.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_1106_4198_gb300 as onmf
from helpers import problem

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (F, K, n, n_inner, precision); K > 128 runs the cluster h-solve
CASES = [(513, 100, 300, 10, onmf.ONMF_FP32),
         (129, 8, 77, 5, onmf.ONMF_MIXED),
         (513, 100, 200, 10, onmf.ONMF_MIXED),
         (513, 256, 150, 10, onmf.ONMF_MIXED)]


def regular(W0, V, n_inner, precision, eps=1e-12):
    import torch
    K, F = W0.shape
    m = onmf.OnlineISNMF(F, K, W0, n_inner=n_inner, precision=precision, eps=eps)
    H = torch.zeros((V.shape[0], K), device="cuda")
    obj = m.project(torch.as_tensor(V).cuda(), H, want_obj=True)
    m.close()
    return H.cpu().numpy(), obj


class StaticCall:
    """Device buffers of one static call, allocated before the call so that
    the call itself can be checked for allocations."""

    def __init__(self, W0, V):
        import torch
        self.W = torch.as_tensor(W0).cuda()
        self.V = torch.as_tensor(V).cuda()
        self.H = torch.full((V.shape[0], W0.shape[0]), -1.0, device="cuda")
        self.obj = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.err = torch.full((1,), -1, dtype=torch.int32, device="cuda")

    def run(self, n_inner, precision, eps=1e-12):
        onmf.onmf_project_static(self.W, self.V, self.H, self.obj, eps=eps,
                                 n_inner=n_inner, precision=precision,
                                 err_out=self.err)

    def results(self):
        import torch
        torch.cuda.synchronize()
        return self.H.cpu().numpy(), float(self.obj.item()), int(self.err.item())


def test_static_projection_equals_allocating_projection_twice():
    for F, K, n, n_in, prec in CASES:
        V, W0 = problem(F, K, n, seed=99)
        Hr, objr = regular(W0, V, n_in, prec)
        for call in range(2):  # the second call sees the first one's scratch
            c = StaticCall(W0, V)
            c.run(n_in, prec)
            Hs, objs, err = c.results()
            print("F=%d K=%d n=%d prec=%d call %d: max |dH| %.3e, obj %r vs %r, err %d"
                  % (F, K, n, prec, call, np.abs(Hs - Hr).max(), objs, objr, err))
            assert err == 0
            assert np.array_equal(Hs, Hr), (F, K, prec, call)
            assert objs == objr, (F, K, prec, call, objs, objr)


def test_second_call_allocates_no_device_memory():
    """Free device memory (cudaMemGetInfo) is the same before and after a
    call that follows a warm-up call of the same shape: the first call of a
    shape may load its kernels' code, later ones allocate nothing."""
    import torch
    for F, K, n, n_in, prec in CASES:
        V, W0 = problem(F, K, n, seed=7)
        c = StaticCall(W0, V)
        c.run(n_in, prec)  # warm-up: kernels of this shape loaded
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        c.run(n_in, prec)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        _, _, err = c.results()
        print("F=%d K=%d prec=%d: free %d -> %d" % (F, K, prec, free0, free1))
        assert err == 0
        assert free1 == free0, (F, K, prec, free0 - free1)


def test_static_projection_reports_invalid_frames():
    """A NaN frame is flagged by the kernels' input check in err_out
    (ONMF_DEVERR_INPUT); a clean call afterwards clears it."""
    F, K, n = 129, 8, 40
    V, W0 = problem(F, K, n, seed=5)
    bad = V.copy()
    bad[17, 3] = np.nan
    for prec in (onmf.ONMF_FP32, onmf.ONMF_MIXED):
        c = StaticCall(W0, bad)
        c.run(5, prec)
        _, _, err = c.results()
        assert err & onmf.ONMF_DEVERR_INPUT, (prec, err)
        c = StaticCall(W0, V)
        c.run(5, prec)
        _, _, err = c.results()
        assert err == 0, (prec, err)


def test_static_projection_rejects_oversized_requests():
    """F = 8192, K = 256 in FP32: the row-major image of W alone needs 8 MiB,
    more than the 4 MiB array. The buffers match the sizes passed, so even
    a call that got past the size check would read only memory that exists."""
    import torch
    F, K, n = 8192, 256, 8
    W = torch.ones((K, F), device="cuda") / F
    V = torch.ones((n, F), device="cuda")
    H = torch.zeros((n, K), device="cuda")
    with pytest.raises(onmf.OnmfError) as e:
        onmf.onmf_project_static(W, V, H, precision=onmf.ONMF_FP32)
    assert e.value.status == 1  # ONMF_EINVAL


FRESH = r"""
import json, sys
sys.path.insert(0, %(root)r)
sys.path.insert(0, %(tests)r)
import numpy as np, torch
import paper_1106_4198_gb300 as onmf
from helpers import problem
out = []
for F, K, n, n_in, prec in %(cases)r:
    V, W0 = problem(F, K, n, seed=3)
    W = torch.as_tensor(W0).cuda(); Vd = torch.as_tensor(V).cuda()
    H = torch.full((n, K), -1.0, device="cuda")
    obj = torch.zeros(1, dtype=torch.float64, device="cuda")
    err = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    # the static entry point is this process's first call into the library
    onmf.onmf_project_static(W, Vd, H, obj, n_inner=n_in, precision=prec, err_out=err)
    torch.cuda.synchronize()
    Hs, objs = H.cpu().numpy(), float(obj.item())
    m = onmf.OnlineISNMF(F, K, W0, n_inner=n_in, precision=prec)
    Hr = torch.zeros((n, K), device="cuda")
    objr = m.project(Vd, Hr, want_obj=True)
    m.close()
    out.append(dict(F=F, K=K, prec=prec, err=int(err.item()),
                    equal=bool(np.array_equal(Hs, Hr.cpu().numpy())) and objs == objr))
print("RESULT " + json.dumps(out))
"""


def test_first_call_in_a_fresh_process():
    code = FRESH % dict(root=ROOT, tests=os.path.join(ROOT, "tests"),
                        cases=[CASES[1], CASES[0]])
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       timeout=600)
    print(r.stdout[-2000:], r.stderr[-2000:])
    assert r.returncode == 0
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    assert len(res) == 2
    for x in res:
        assert x["err"] == 0 and x["equal"], x
