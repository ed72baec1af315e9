"""Failure detection on the GPU without a GPU fault: every device-side wait
of the library is bounded by a time limit, after which the kernel flags a
timeout, releases what it holds and returns, and the host sees
ONMF_ETIMEOUT with the CUDA context still usable.

onmf_selftest_wait drives each wait on a condition that nothing satisfies
(a grid barrier expecting one CTA more than the grid has, an mbarrier that
nothing arrives on, the same while holding tensor memory). Afterwards the
normal path must still run and match its result from before."""
import numpy as np
import pytest

import paper_1106_4198_gb300 as onmf
from helpers import cuda, problem

pytestmark = pytest.mark.gpu

LIMIT_NS = 2_000_000_000


def small_run():
    F, K = 129, 8
    V, W0 = problem(F, K, 200, seed=3)
    m = onmf.OnlineISNMF(F, K, W0, beta=50, n_inner=3, precision=onmf.ONMF_MIXED)
    m.push(cuda(V))
    m.sync()
    W = m.W()
    m.close()
    return W


@pytest.mark.parametrize("which", [0, 1, 2])
def test_bounded_wait_times_out_and_context_survives(which):
    before = small_run()
    st, el = onmf.onmf_selftest_wait(which)
    print("wait %d: status %s after %.3f s" % (which, onmf.onmf_status_string(st), el * 1e-9))
    assert st == onmf.ONMF_ETIMEOUT
    # the wait ran to its limit, not much past it
    assert LIMIT_NS <= el < 3 * LIMIT_NS
    after = small_run()
    assert np.array_equal(before, after)

