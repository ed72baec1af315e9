"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage of arXiv:1106.4198 it checks. None of them
compares the oracle with itself: the expected values are closed forms,
brute-force minima, identities the paper states, or invariants of the
arithmetic (power-of-two scaling is exact in IEEE floating point).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def rng(seed):
    return np.random.default_rng(seed)


def rand_W(r, K, F, normalize=True):
    W = r.gamma(1.0, 1.0, size=(K, F))
    if normalize:
        W /= W.sum(axis=1, keepdims=True)
    return W


def rand_V(r, n, F, lo=0.05):
    return (r.gamma(1.0, 1.0, size=(n, F)) + lo).astype(np.float32)


# ---------------------------------------------------------------- P1: d_IS


def test_dis_golden_values():
    """Section 2.1: d_IS(y,x) = sum(y/x - log(y/x) - 1), hand values."""
    g = json.load(open(GOLDEN))["dis_scalar"]
    for c in g["cases"]:
        d = oracle.dis([c["y"]], [c["x"]])
        assert d == pytest.approx(c["d"], rel=1e-15, abs=1e-17)


def test_dis_nonnegative_zero_iff_equal():
    """Section 2.1: d_IS >= 0 with equality at y = x."""
    r = rng(1)
    y = r.gamma(1.0, 1.0, 1000) + 1e-3
    x = r.gamma(1.0, 1.0, 1000) + 1e-3
    for i in range(1000):
        d = oracle.dis(y[i:i + 1], x[i:i + 1])
        assert d >= 0.0
    assert oracle.dis(y, y) == 0.0
    # a perturbation of one entry gives a strictly positive divergence
    x2 = y.copy()
    x2[17] *= 1.001
    assert oracle.dis(y, x2) > 0.0


def test_dis_scale_invariance():
    """d_IS(l*y, l*x) = d_IS(y, x): the IS divergence is scale invariant."""
    r = rng(2)
    y = r.gamma(1.0, 1.0, 513) + 1e-3
    x = r.gamma(1.0, 1.0, 513) + 1e-3
    d = oracle.dis(y, x)
    for lam in (1e-6, 0.37, 4.0, 1e5):
        assert oracle.dis(lam * y, lam * x) == pytest.approx(d, rel=1e-12)
    # powers of two are exact
    assert oracle.dis(8.0 * y, 8.0 * x) == d


def test_objective_matches_definition_small():
    """Eq. (is_nmf) with eps: (1/N) sum_n d_IS(eps+v_n, eps+W h_n), on a
    2x2x2 case written out by hand."""
    V = np.array([[1.0, 2.0], [3.0, 0.5]], dtype=np.float32)  # frames
    W = np.array([[0.5, 0.5], [0.25, 0.75]])  # rows = columns of W
    H = np.array([[1.0, 2.0], [0.5, 4.0]])  # frames x K
    eps = 0.25
    tot = 0.0
    for n in range(2):
        for f in range(2):
            x = eps + W[0, f] * H[n, 0] + W[1, f] * H[n, 1]
            y = eps + float(V[n, f])
            tot += y / x - math.log(y / x) - 1.0
    assert oracle.objective(V, W, H, eps) == pytest.approx(tot / 2, rel=1e-14)


# ------------------------------------------------- P2/P3: h-solve closed form


def test_hsolve_k1_golden_trajectory():
    """K = 1 closed form (Section 2.1 MM step): h_n = sqrt(h_{n-1} h*)."""
    g = json.load(open(GOLDEN))["hsolve_k1"]
    W = np.array([g["w"]])
    v = np.array(g["v"], dtype=np.float32)
    traj = g["trajectory_gamma_half"]
    for n in range(len(traj)):
        h = oracle.hsolve(W, v, eps=0.0, gamma=0.5, n_in=n)
        assert h[0] == pytest.approx(traj[n], rel=1e-14)


def test_hsolve_k1_closed_form_random():
    """K = 1, eps = 0: h* = (1/F) sum v/w; with gamma = 1/2 the log-distance
    to h* halves every step; with gamma = 1 one step reaches h*."""
    r = rng(3)
    F = 37
    w = r.gamma(1.0, 1.0, F) + 0.1
    v = (r.gamma(1.0, 1.0, F) + 0.1).astype(np.float32)
    W = w[None, :]
    hstar = np.mean(v.astype(np.float64) / w)
    h0 = v.astype(np.float64).sum() / w.sum()
    for n in (1, 2, 5, 12):
        h, tr = oracle.hsolve(W, v, eps=0.0, gamma=0.5, n_in=n, trace=True)
        expect = math.log(hstar) + (math.log(h0) - math.log(hstar)) / 2**n
        assert math.log(h[0]) == pytest.approx(expect, rel=1e-12, abs=1e-13)
    h = oracle.hsolve(W, v, eps=0.0, gamma=1.0, n_in=1)
    assert h[0] == pytest.approx(hstar, rel=1e-13)
    # h* is the minimizer of d_IS(v, w h)
    d = lambda hh: oracle.dis(v.astype(np.float64), w * hh)
    assert d(hstar) <= d(hstar * 1.001) and d(hstar) <= d(hstar * 0.999)


def test_hsolve_block_diagonal_full_size():
    """F = 513, K = 100 with disjoint row supports per column and eps = 0:
    the h-solve decouples into K copies of the K = 1 closed form, so every
    h_k follows log h_k(n) = log h*_k + (log h0 - log h*_k)/2^n exactly."""
    r = rng(4)
    F, K, n_in = 513, 100, 10
    owner = np.arange(F) % K
    W = np.zeros((K, F))
    W[owner, np.arange(F)] = r.gamma(1.0, 1.0, F) + 0.05
    v = (r.gamma(1.0, 1.0, F) + 0.05).astype(np.float32)
    h = oracle.hsolve(W, v, eps=0.0, gamma=0.5, n_in=n_in)
    h0 = v.astype(np.float64).sum() / W.sum()
    for k in range(K):
        sel = owner == k
        hstar = np.mean(v[sel].astype(np.float64) / W[k, sel])
        expect = math.log(hstar) + (math.log(h0) - math.log(hstar)) / 2**n_in
        assert math.log(h[k]) == pytest.approx(expect, rel=1e-12, abs=1e-12)


# ------------------------------------------- P4: F = K = 2 brute force


def _dis2(v, W, h):
    x = W.T @ h
    return oracle.dis(v.astype(np.float64), x)


def test_hsolve_2x2_interior_solution():
    """If W^{-1} v >= 0, the minimum of d_IS(v, W h) is 0 at h = W^{-1} v,
    and the MM iteration converges there (W diagonally dominant, so the
    iteration contracts quickly; nearly collinear columns converge slowly)."""
    r = rng(5)
    for trial in range(5):
        W = np.eye(2) + 0.3 * r.random((2, 2))
        htrue = r.gamma(2.0, 1.0, size=2) + 0.2
        v = (W.T @ htrue).astype(np.float32)
        hexact = np.linalg.solve(W.T, v.astype(np.float64))
        assert np.all(hexact > 0)
        h = oracle.hsolve(W, v, eps=0.0, gamma=0.5, n_in=2000)
        assert np.allclose(h, hexact, rtol=1e-6)
        assert _dis2(v, W, h) < 1e-12


def test_hsolve_2x2_face_solution_brute_force():
    """If W^{-1} v has a negative entry, the constrained minimum lies on a
    face h_k = 0. Compare the MM result with the closed-form face minima and
    with a grid search over [0, hmax]^2."""
    W = np.array([[1.0, 0.1], [0.2, 1.0]])  # rows: columns of W
    v = np.array([1.0, 0.05], dtype=np.float32)
    vd = v.astype(np.float64)
    hexact = np.linalg.solve(W.T, vd)
    assert np.any(hexact < 0)
    faces = []
    for k in range(2):
        hk = np.mean(vd / W[k])
        h = np.zeros(2)
        h[k] = hk
        faces.append(_dis2(v, W, h))
    dface = min(faces)
    # grid search (brute force) over the quadrant
    best = np.inf
    for a in np.linspace(0.0, 2.0, 401):
        for b in np.linspace(0.0, 0.5, 201):
            if a == 0.0 and b == 0.0:
                continue
            best = min(best, _dis2(v, W, np.array([a, b])))
    assert best >= dface - 1e-9
    h = oracle.hsolve(W, v, eps=0.0, gamma=0.5, n_in=2000)
    dmm = _dis2(v, W, h)
    assert dmm >= dface - 1e-12
    assert dmm <= dface + 1e-3 * max(dface, 1e-12)


# ----------------------------------------------------- P5: monotone descent


def test_hsolve_monotone_descent():
    """Section 2.1: the MM step is a descent step; with eps > 0 the fixed
    eps component does not break the majorization."""
    r = rng(6)
    F, K = 64, 8
    W = rand_W(r, K, F)
    for trial in range(10):
        v = rand_V(r, 1, F)[0]
        _, tr = oracle.hsolve(W, v, eps=1e-12, gamma=0.5, n_in=60, trace=True)
        assert np.all(np.diff(tr) <= 1e-12 * tr[:-1])
        assert tr[-1] < tr[0]


def test_batch_monotone_descent():
    """Section 2.1: batch IS-NMF alternates descent steps in H and W, so the
    objective is non-increasing after every half step."""
    r = rng(7)
    F, K, N = 40, 5, 120
    V = rand_V(r, N, F)
    W = rand_W(r, K, F)
    H = oracle.batch_h0(V, W, eps=1e-12)
    prev = oracle.objective(V, W, H, 1e-12)
    for it in range(15):
        for which in (1, 2):
            W, H, obj = oracle.batch(V, W, H, eps=1e-12, gamma=0.5, n_iter=1,
                                     which=which)
            assert obj[0] <= prev * (1 + 1e-12)
            prev = obj[0]


# ---------------------------------------------------- P6: dictionary step


def test_sqrt_ab_minimizes_aux():
    """Eq. (aux_fun0): W = sqrt(A/B) minimizes A/W + B W entrywise."""
    r = rng(8)
    A = r.gamma(1.0, 1.0, 500) + 1e-3
    B = r.gamma(1.0, 1.0, 500) + 1e-3
    W = np.sqrt(A / B)
    g = lambda w: A / w + B * w
    for d in (1e-4, 1e-2, 0.3):
        assert np.all(g(W) <= g(W * (1 + d)))
        assert np.all(g(W) <= g(W * (1 - d)))


def test_stats_step_rescale_keeps_sqrt_ab():
    """Section 2.3 "Rescaling W": after W/s, A/s, B*s the relation
    W = sqrt(A/B) still holds and every column of W sums to 1."""
    r = rng(9)
    F, K, n = 50, 6, 40
    V = rand_V(r, n, F)
    W = rand_W(r, K, F)
    H = r.gamma(1.0, 1.0, size=(n, K)) + 0.01
    A = r.gamma(1.0, 1.0, size=(K, F))
    B = r.gamma(1.0, 1.0, size=(K, F))
    W2, A2, B2, _ = oracle.stats_step(V, W, A, B, H, eps=1e-12, rho=0.9)
    assert np.allclose(W2, np.sqrt(A2 / B2), rtol=1e-14)
    assert np.allclose(W2.sum(axis=1), 1.0, rtol=1e-14)


def test_stats_step_matches_written_out_formulas():
    """Algorithm 1, statistics lines, written out for one (f, k) entry on a
    tiny case: a_fk = W_fk^2 sum_j y_fj/x_fj^2 h_kj, b_fk = sum_j h_kj/x_fj,
    A <- rho A + a, W = sqrt(A/B) before the rescale."""
    r = rng(10)
    F, K, n = 3, 2, 4
    V = rand_V(r, n, F)
    W = rand_W(r, K, F)
    H = r.gamma(1.0, 1.0, size=(n, K)) + 0.1
    A = r.gamma(1.0, 1.0, size=(K, F))
    B = r.gamma(1.0, 1.0, size=(K, F))
    eps, rho = 0.01, 0.5
    W2, A2, B2, loss = oracle.stats_step(V, W, A, B, H, eps=eps, rho=rho,
                                         normalize=False)
    for f in range(F):
        for k in range(K):
            a = b = 0.0
            for j in range(n):
                x = eps + sum(W[kk, f] * H[j, kk] for kk in range(K))
                y = eps + float(V[j, f])
                a += y / x**2 * H[j, k]
                b += H[j, k] / x
            a *= W[k, f] ** 2
            Ae = rho * A[k, f] + a
            Be = rho * B[k, f] + b
            assert A2[k, f] == pytest.approx(Ae, rel=1e-13)
            assert B2[k, f] == pytest.approx(Be, rel=1e-13)
            assert W2[k, f] == pytest.approx(math.sqrt(Ae / Be), rel=1e-13)
    # literal reading of Algorithm 1: A <- A + rho * a
    W3, A3, B3, _ = oracle.stats_step(V, W, A, B, H, eps=eps, rho=rho,
                                      normalize=False, rho_on_new=True)
    assert np.allclose(A3 - A, rho * (A2 - rho * A), rtol=1e-12)


def test_stats_step_guard_zero_b():
    """Guard: entries with B = 0 keep their W value (W is never 0/0)."""
    F, K, n = 4, 2, 3
    V = np.ones((n, F), dtype=np.float32)
    W = np.full((K, F), 0.25)
    H = np.zeros((n, K))
    H[:, 0] = 1.0  # column 1 of H is zero -> b_{:,1} = 0
    A = np.zeros((K, F))
    B = np.zeros((K, F))
    W2, A2, B2, _ = oracle.stats_step(V, W, A, B, H, eps=1e-12, rho=1.0,
                                      normalize=False)
    assert np.all(W2[1] == 0.25)
    assert np.all(B2[1] == 0.0)


# ------------------------------------------------ P7: online equals batch


def test_online_step_equals_batch_w_step_fixed_h():
    """Section 2.3 "Overview": with A0 = B0 = 0 and the whole set in one
    minibatch, the dictionary step equals the batch W update."""
    r = rng(11)
    F, K, N = 30, 4, 64
    V = rand_V(r, N, F)
    W0 = rand_W(r, K, F)
    H0 = oracle.batch_h0(V, W0, eps=1e-12)
    _, H1, _ = oracle.batch(V, W0, H0, n_iter=1, which=1)
    Wb, _, _ = oracle.batch(V, W0, H1, n_iter=1, which=2)
    Wo, _, _, _ = oracle.stats_step(V, W0, np.zeros((K, F)), np.zeros((K, F)),
                                    H1, eps=1e-12, rho=0.0)
    assert np.max(np.abs(Wo - Wb) / Wb) < 1e-13


def test_online_r0_full_batch_equals_first_batch_iteration():
    """Section 2.3 "Overview": beta = N and r = 0 make the online algorithm
    the batch algorithm; with one inner step the first online update equals
    the first batch iteration from the same start point."""
    r = rng(12)
    F, K, N = 25, 3, 48
    V = rand_V(r, N, F)
    W0 = rand_W(r, K, F)
    out = oracle.online_pass(V, W0, beta=N, n_in=1, eps=1e-12, gamma=0.5,
                             r=0.0, n_ref=N)
    H0 = oracle.batch_h0(V, W0, eps=1e-12)
    Wb, Hb, _ = oracle.batch(V, W0, H0, n_iter=1)
    assert np.max(np.abs(out["W"] - Wb) / Wb) < 1e-13
    # online keeps h from before the rescale; batch scales row k of H by s_k
    s = Hb[0] / out["H"][0]
    assert np.allclose(Hb, out["H"] * s[None, :], rtol=1e-12)


# ------------------------------------------------- P11: warm restarts


def test_warm_restart_from_fresh_start_point_is_the_fresh_restart():
    """Section 2.3 "Fresh or warm restarts": a warm start from the
    fresh-restart point itself reproduces the fresh restart, bit for bit
    (one minibatch, so both use W0)."""
    r = rng(41)
    F, K, N = 20, 3, 30
    V = rand_V(r, N, F)
    W0 = rand_W(r, K, F)
    fresh = oracle.online_pass(V, W0, beta=N, n_in=4)
    warm = oracle.online_pass(V, W0, beta=N, n_in=4, H_init=oracle.batch_h0(V, W0))
    for k in ("W", "A", "B", "H"):
        assert np.array_equal(fresh[k], warm[k]), k
    assert fresh["loss_sum"] == warm["loss_sum"]


def test_warm_passes_over_the_whole_set_are_batch_iterations():
    """With the whole finite set as one minibatch, r = 0, one h update per
    visit and warm restarts, every pass is one batch MU cycle (Section 2.1)
    from the same (W, H); without the rescale the kept H is the batch H."""
    r = rng(42)
    F, K, N = 24, 3, 40
    V = rand_V(r, N, F)
    W0 = rand_W(r, K, F)
    H = r.gamma(1.0, 1.0, size=(N, K)) + 0.1
    W, A, B = W0, None, None
    Hk = H.copy()
    for _ in range(3):
        out = oracle.online_pass(V, W, A, B, beta=N, n_in=1, r=0.0, n_ref=N,
                                 normalize=False, H_init=Hk)
        W, A, B, Hk = out["W"], out["A"], out["B"], out["H"]
    Wb, Hb, _ = oracle.batch(V, W0, H, n_iter=3, normalize=False)
    assert np.max(np.abs(W - Wb) / Wb) < 1e-12
    assert np.max(np.abs(Hk - Hb) / Hb) < 1e-12


# ------------------------------------------- P8: scale equivariance (exact)


def test_scale_equivariance_bitwise():
    """With eps = 0, V -> 4V gives H -> 4H and leaves W, A, B and the loss
    unchanged, bit for bit (multiplying by a power of two is exact and every
    ratio y/x, y/x^2 * h, h/x is invariant)."""
    r = rng(13)
    F, K, N = 33, 5, 60
    V = rand_V(r, N, F)
    W0 = rand_W(r, K, F)
    a = oracle.online_pass(V, W0, beta=20, n_in=4, eps=0.0)
    b = oracle.online_pass(4 * V, W0, beta=20, n_in=4, eps=0.0)
    assert np.array_equal(a["W"], b["W"])
    assert np.array_equal(a["A"], b["A"])
    assert np.array_equal(a["B"], b["B"])
    assert np.array_equal(4 * a["H"], b["H"])
    assert a["loss_sum"] == b["loss_sum"]


# ---------------------------------------------------- P9: fixed point


def test_noiseless_fixed_point():
    """With V = W* H* exactly (no noise), L1-normalized W* and the true H*,
    W* is a fixed point of the dictionary step: P = Q = 1/X, so
    A = W*^2 o B and sqrt(A/B) = W*. Dyadic values keep V exact in float32."""
    r = rng(14)
    F, K, N = 8, 3, 20
    Wst = np.zeros((K, F))
    for k in range(K):
        c = r.integers(1, 8, size=F).astype(np.float64)
        c[-1] += 64 - c.sum() if c.sum() < 64 else 0
        c *= 64.0 / c.sum() if c.sum() != 64 else 1.0
        Wst[k] = c / 64.0
    Wst /= Wst.sum(axis=1, keepdims=True)
    Hst = r.integers(1, 9, size=(N, K)).astype(np.float64)
    V = (Hst @ Wst).astype(np.float32)
    assert np.array_equal(V.astype(np.float64), Hst @ Wst)
    W2, _, _, loss = oracle.stats_step(V, Wst, np.zeros((K, F)), np.zeros((K, F)),
                                       Hst, eps=0.0, rho=1.0)
    assert np.max(np.abs(W2 - Wst) / Wst) < 1e-14
    assert abs(loss) < 1e-12


# --------------------------------------------- P10: order and split invariance


def test_minibatch_permutation_invariance():
    """A and B after a minibatch are sums over its frames, so permuting the
    frames inside the minibatch changes them only by rounding."""
    r = rng(15)
    F, K, n = 40, 6, 30
    V = rand_V(r, n, F)
    W0 = rand_W(r, K, F)
    a = oracle.online_pass(V, W0, beta=n, n_in=3)
    perm = r.permutation(n)
    b = oracle.online_pass(V[perm], W0, beta=n, n_in=3)
    assert np.allclose(a["A"], b["A"], rtol=1e-12)
    assert np.allclose(a["B"], b["B"], rtol=1e-12)
    assert np.allclose(a["W"], b["W"], rtol=1e-12)
    assert np.allclose(a["H"][perm], b["H"], rtol=1e-12)


def test_split_pass_and_restore_are_bitwise_identical():
    """The state of Algorithm 1 is (W, A, B): processing N frames in one pass
    equals two passes that hand the state over (save/restore)."""
    r = rng(16)
    F, K, N, beta = 21, 4, 100, 10
    V = rand_V(r, N, F)
    W0 = rand_W(r, K, F)
    full = oracle.online_pass(V, W0, beta=beta, n_in=3)
    h1 = oracle.online_pass(V[:40], W0, beta=beta, n_in=3)
    h2 = oracle.online_pass(V[40:], h1["W"], h1["A"], h1["B"], beta=beta,
                            n_in=3, loss_sum=h1["loss_sum"])
    assert np.array_equal(full["W"], h2["W"])
    assert np.array_equal(full["A"], h2["A"])
    assert np.array_equal(full["B"], h2["B"])
    assert full["loss_sum"] == h2["loss_sum"]


def test_partial_last_minibatch_and_flush():
    """A pass over N = 2.5 beta frames takes two full minibatches; the last
    half minibatch is processed only on flush, with rho = r^(beta'/n_ref)."""
    r = rng(17)
    F, K, beta = 16, 3, 8
    V = rand_V(r, 20, F)
    W0 = rand_W(r, K, F)
    noflush = oracle.online_pass(V, W0, beta=beta, n_in=2, flush=False,
                                 r=0.5, n_ref=16)
    assert noflush["frames"] == 16 and len(noflush["mb_loss"]) == 2
    fl = oracle.online_pass(V, W0, beta=beta, n_in=2, flush=True, r=0.5,
                            n_ref=16)
    assert fl["frames"] == 20 and len(fl["mb_loss"]) == 3
    assert oracle.rho(0.5, 4, 16) == pytest.approx(0.5 ** 0.25, rel=1e-15)
    # the flushed minibatch equals a direct pass over its 4 frames
    last = oracle.online_pass(V[16:], noflush["W"], noflush["A"], noflush["B"],
                              beta=4, n_in=2, r=0.5, n_ref=16)
    assert np.array_equal(last["W"], fl["W"])


def test_forgetting_factor_r0_forgets_past():
    """r = 0 (rho = 0) with the past-scaling reading: A and B after a
    minibatch depend on that minibatch only."""
    r = rng(18)
    F, K, beta = 12, 3, 6
    V = rand_V(r, 12, F)
    W0 = rand_W(r, K, F)
    A0 = r.gamma(1.0, 1.0, size=(K, F))
    B0 = r.gamma(1.0, 1.0, size=(K, F))
    a = oracle.online_pass(V[:6], W0, A0, B0, beta=beta, n_in=2, r=0.0,
                           n_ref=beta)
    b = oracle.online_pass(V[:6], W0, None, None, beta=beta, n_in=2, r=0.0,
                           n_ref=beta)
    assert np.array_equal(a["A"], b["A"]) and np.array_equal(a["W"], b["W"])


def test_project_equals_per_frame_hsolve():
    """Projection (held-out evaluation, Section 3) is the h-solve of each
    frame with W fixed; its objective sum is sum_n d_IS at the solution."""
    r = rng(19)
    F, K, N = 20, 4, 7
    V = rand_V(r, N, F)
    W = rand_W(r, K, F)
    H, s = oracle.project(V, W, n_in=6)
    for n in range(N):
        h = oracle.hsolve(W, V[n], n_in=6)
        assert np.array_equal(h, H[n])
    assert s == pytest.approx(oracle.objective(V, W, H, 1e-12) * N, rel=1e-14)


def test_threads_do_not_change_results():
    """The OpenMP option splits independent frames/rows only."""
    r = rng(20)
    F, K, N = 30, 5, 50
    V = rand_V(r, N, F)
    W0 = rand_W(r, K, F)
    oracle.set_threads(1)
    a = oracle.online_pass(V, W0, beta=25, n_in=3)
    oracle.set_threads(4)
    b = oracle.online_pass(V, W0, beta=25, n_in=3)
    oracle.set_threads(1)
    assert np.array_equal(a["W"], b["W"]) and np.array_equal(a["H"], b["H"])


# ------------------------------- P12: penalties (Section 2.2, "Extensions")
# h penalty lambda * log(a + sum_k h_k) (psi concave increasing), dictionary
# penalty mu * sum W. Pinned by the K = 1 stationary point in closed form, a
# brute-force grid minimum at F = K = 2, the objective recomputed here, and the
# minimizer property of the penalized dictionary step.


def _pen_obj(v, W, h, lam, a):
    """d_IS(v, W h) + lam * log(a + sum h) at eps = 0, evaluated with numpy."""
    y = v.astype(np.float64)
    x = W.T @ h
    return float(np.sum(y / x - np.log(y / x) - 1.0) + lam * np.log(a + h.sum()))


def test_penalized_hsolve_k1_closed_form():
    """K = 1: the objective S/h + F log h + lam log(a + h) (S = sum_f v_f/w_f,
    up to constants) is stationary where F h + lam h^2/(a + h) = S, i.e. at the
    positive root of (F + lam) h^2 + (F a - S) h - S a = 0."""
    r = rng(21)
    F = 50
    W = r.gamma(1.0, 1.0, size=(1, F)) + 0.05
    v = rand_V(r, 1, F)[0]
    S = float(np.sum(v.astype(np.float64) / W[0]))
    for lam, a in ((0.5, 1.0), (5.0, 0.2), (50.0, 3.0)):
        qa, qb, qc = F + lam, F * a - S, -S * a
        hstar = (-qb + math.sqrt(qb * qb - 4 * qa * qc)) / (2 * qa)
        h = oracle.hsolve(W, v, eps=0.0, gamma=0.5, n_in=400, h_penalty=lam, h_penalty_a=a)
        assert abs(h[0] - hstar) <= 1e-10 * hstar, (lam, a, h[0], hstar)
    # no penalty: the plain K = 1 solution S / F
    h = oracle.hsolve(W, v, eps=0.0, gamma=0.5, n_in=400)
    assert abs(h[0] - S / F) <= 1e-10 * S / F


def test_penalized_hsolve_2x2_brute_force():
    """F = K = 2 with the h penalty: the MM iterate reaches the minimum that
    a fine grid search of the penalized objective finds."""
    W = np.array([[1.0, 0.3], [0.2, 0.9]])
    v = np.array([1.2, 0.8], dtype=np.float32)
    lam, a = 0.6, 0.5
    best, arg = np.inf, None
    for x0 in np.linspace(1e-3, 2.0, 400):
        for x1 in np.linspace(1e-3, 2.0, 400):
            o = _pen_obj(v, W, np.array([x0, x1]), lam, a)
            if o < best:
                best, arg = o, (x0, x1)
    h = oracle.hsolve(W, v, eps=0.0, gamma=0.5, n_in=5000, h_penalty=lam, h_penalty_a=a)
    o = _pen_obj(v, W, h, lam, a)
    assert o <= best + 1e-9
    assert abs(h[0] - arg[0]) <= 0.01 and abs(h[1] - arg[1]) <= 0.01
    # the penalty moves the minimum: the plain solution W^{-T} v is not it
    h0 = np.linalg.solve(W.T, v.astype(np.float64))
    assert _pen_obj(v, W, h0, lam, a) > o + 1e-6


def test_penalized_hsolve_descent_and_trace():
    """The tangent majorization of the concave penalty keeps every MM step a
    descent step of the penalized objective; the oracle's trace is that
    objective (recomputed here at the last iterate)."""
    r = rng(22)
    F, K = 64, 8
    W = rand_W(r, K, F)
    for lam, a in ((1.0, 1.0), (20.0, 0.1)):
        for trial in range(5):
            v = rand_V(r, 1, F)[0]
            h, tr = oracle.hsolve(W, v, eps=0.0, gamma=0.5, n_in=60, trace=True,
                                  h_penalty=lam, h_penalty_a=a)
            assert np.all(np.diff(tr) <= 1e-12 * np.abs(tr[:-1]))
            assert tr[-1] < tr[0]
            assert abs(tr[-1] - _pen_obj(v, W, h, lam, a)) <= 1e-10 * abs(tr[-1])


def test_h_penalty_shrinks_the_activations():
    """A larger lambda gives a smaller sum_k h_k at the same frame."""
    r = rng(23)
    F, K = 64, 8
    W = rand_W(r, K, F)
    v = rand_V(r, 1, F)[0]
    sums = [oracle.hsolve(W, v, eps=0.0, n_in=300, h_penalty=lam, h_penalty_a=1.0).sum()
            for lam in (0.0, 1.0, 10.0, 100.0)]
    assert all(s1 > s2 for s1, s2 in zip(sums[:-1], sums[1:])), sums


def test_w_penalty_dictionary_step_minimizes_aux():
    """With mu * sum W the dictionary step minimizes A/W + (B + mu) W
    entrywise; mu = 0 is the plain step, bit for bit."""
    r = rng(24)
    F, K, n = 40, 5, 30
    V = rand_V(r, n, F)
    W = rand_W(r, K, F)
    H = r.gamma(1.0, 1.0, size=(n, K)) + 0.01
    A = r.gamma(1.0, 1.0, size=(K, F))
    B = r.gamma(1.0, 1.0, size=(K, F))
    mu = 0.7
    W2, A2, B2, _ = oracle.stats_step(V, W, A, B, H, eps=1e-12, rho=1.0, normalize=False,
                                      w_penalty=mu)
    g = lambda w: A2 / w + (B2 + mu) * w
    for d in (1e-4, 1e-2, 0.3):
        assert np.all(g(W2) <= g(W2 * (1 + d)))
        assert np.all(g(W2) <= g(W2 * (1 - d)))
    Wp, Ap, Bp, lp = oracle.stats_step(V, W, A, B, H, eps=1e-12, rho=1.0, normalize=False)
    Wz, Az, Bz, lz = oracle.stats_step(V, W, A, B, H, eps=1e-12, rho=1.0, normalize=False,
                                       w_penalty=0.0)
    assert np.array_equal(Wp, Wz) and np.array_equal(Ap, Az) and lp == lz
