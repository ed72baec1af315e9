"""The allocation-free projection (onmf_project_static), called through the
C ABI, against the regular projection (onmf_project) on the same inputs.

onmf_project_static serves callers that cannot allocate device memory (a
real-time audio callback, a host with a fixed memory arena). It keeps its
scratch in one static device array shared by all calls, so the test makes
two calls in a row with different shapes and precisions (the second must
not see the first's leftovers) and checks each against the allocating path
within the FP32 tolerance of the parity tests (1e-5, norm-wise relative).
It runs alone in a fresh process as well as after the other tests."""
import numpy as np
import pytest

import paper_1106_4198_gb300 as onmf
from helpers import problem, relerr

pytestmark = pytest.mark.gpu


def regular(W0, V, n_inner, precision, eps=1e-12):
    import torch
    K, F = W0.shape
    m = onmf.OnlineISNMF(F, K, W0, n_inner=n_inner, precision=precision, eps=eps)
    H = torch.zeros((V.shape[0], K), device="cuda")
    obj = m.project(torch.as_tensor(V).cuda(), H, want_obj=True)
    m.close()
    return H.cpu().numpy(), obj


def static(W0, V, n_inner, precision, eps=1e-12):
    import torch
    K, F = W0.shape
    W = torch.as_tensor(W0).cuda()
    Vd = torch.as_tensor(V).cuda()
    H = torch.full((V.shape[0], K), -1.0, device="cuda")
    obj = torch.zeros(1, dtype=torch.float64, device="cuda")
    onmf.onmf_project_static(W, Vd, H, obj, eps=eps, n_inner=n_inner,
                             precision=precision)
    torch.cuda.synchronize()
    return H.cpu().numpy(), float(obj.item())


def test_static_projection_matches_allocating_projection_twice():
    cases = [(513, 100, 300, 10, onmf.ONMF_FP32),
             (129, 8, 77, 5, onmf.ONMF_MIXED),
             (513, 100, 200, 10, onmf.ONMF_MIXED),
             (513, 256, 150, 10, onmf.ONMF_MIXED)]  # K > 128: the cluster h-solve
    for F, K, n, n_in, prec in cases:
        V, W0 = problem(F, K, n, seed=99)
        Hr, objr = regular(W0, V, n_in, prec)
        Hs, objs = static(W0, V, n_in, prec)
        e = relerr(Hs, Hr)
        eo = abs(objs - objr) / abs(objr)
        print("F=%d K=%d n=%d prec=%d: H rel err %.2e, obj rel err %.2e"
              % (F, K, n, prec, e, eo))
        assert e <= 1e-5 and eo <= 1e-5


def test_static_projection_rejects_oversized_requests():
    import torch
    F, K = 513, 256
    W = torch.ones((K, F), device="cuda") / F
    V = torch.ones((8, F), device="cuda")
    # the FP32 image of W alone needs 4*F*K = 525 KB; 40 M frames of loss
    # slots (5 M doubles) exceed the 4 MiB array
    with pytest.raises(onmf.OnmfError) as e:
        onmf.lib()  # ensure loaded
        st = onmf.lib().onmf_project_static(W.data_ptr(), F, K, V.data_ptr(), F,
                                            40_000_000, None, K, 1e-12, 0.5, 10,
                                            onmf.ONMF_FP32, None, None)
        onmf._check(st, "onmf_project_static")
    assert e.value.status == 1  # ONMF_EINVAL
