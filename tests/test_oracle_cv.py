"""Pins of the oracle's control-variate estimator.

Y_cv = Y - sum_{j < kappa} G(s_j, X_j) . sqrt(2) dW_j with G any model of the
solution's gradient, evaluated at the start of each sub-step. The sum is a
martingale stopped at a bounded time, so E[Y_cv] = E[Y] for every model; with
the exact gradient of the heat problem the per-path variance collapses down
to the sub-step discretisation's share.
"""
import math

import numpy as np
import pytest

import workloads as W


def _heat_problem(oracle_mod):
    xi0, eta0 = W.heat65_fields()
    faces = np.zeros(oracle_mod.faces_len(65, 65))
    return oracle_mod.Problem(W.w_const(65), xi0, eta0, faces)


def test_zero_model_is_the_plain_estimator(oracle_mod):
    n = 33
    P = oracle_mod.Problem(W.w_smooth_random(n, 3), *W.identity_fields(n))
    xs, ys = np.array([0.5, 0.1]), np.array([0.5, 0.7])
    kw = dict(dt=1e-3, Dt=0.02, seed=4, record=True)
    a = oracle_mod.interface_mc(P, xs, ys, 300, **kw)
    b = oracle_mod.interface_mc(P, xs, ys, 300, cv_table=np.zeros((3, n, n, 4)), **kw)
    for k in ("score_xi", "score_eta", "steps", "code", "mean_xi", "se_xi"):
        np.testing.assert_array_equal(a[k], b[k])


def test_any_model_leaves_the_mean_unbiased(oracle_mod):
    # a smooth model unrelated to the solution: E[sum G . sqrt(2) dW] = 0
    n = 65
    P = oracle_mod.Problem(W.w_front(n, 0.1), *W.identity_fields(n))
    X, Y = W.grid(n)
    S = 4
    T = np.zeros((S, n, n, 4))
    for q in range(S):
        T[q, ..., 0] = 2.0 * np.sin(3 * X + q) * np.cos(2 * Y)
        T[q, ..., 1] = 1.5 + np.cos(5 * X * Y)
        T[q, ..., 2] = -3.0 * X * Y + q
        T[q, ..., 3] = np.sin(4 * Y - X)
    xs, ys = np.array([0.5, 0.3, 0.08]), np.array([0.5, 0.62, 0.4])
    kw = dict(dt=2e-4, Dt=1e-2, seed=8, record=True)
    N = 20000
    a = oracle_mod.interface_mc(P, xs, ys, N, **kw)
    b = oracle_mod.interface_mc(P, xs, ys, N, cv_table=T, **kw)
    np.testing.assert_array_equal(a["code"], b["code"])     # the model never moves a path
    for f in ("xi", "eta"):
        D = (b["score_" + f] - a["score_" + f]).reshape(3, N)
        assert np.all(D.std(axis=1) > 1e-3)                 # the term is really there
        z = D.mean(axis=1) / (D.std(axis=1, ddof=1) / math.sqrt(N))
        assert np.all(np.abs(z) < 4.0), z


def test_exact_gradient_collapses_the_variance(oracle_mod):
    # heat problem: v(s, x) = exp(-2 pi^2 s) sin(pi x) sin(pi y) (xi) and
    # exp(-5 pi^2 s) sin(pi x) sin(2 pi y) (eta), s the time left in the step;
    # one slice per sub-step holds grad v at s_j = Dt - j dt
    P = _heat_problem(oracle_mod)
    n, dt, Dt = 65, 5e-4, 0.05
    K = int(round(Dt / dt))
    X, Y = W.grid(n)
    T = np.zeros((K, n, n, 4))
    for j in range(K):
        s = Dt - j * dt
        ex, ee = math.exp(-2 * math.pi ** 2 * s), math.exp(-5 * math.pi ** 2 * s)
        T[j, ..., 0] = ex * math.pi * np.cos(np.pi * X) * np.sin(np.pi * Y)
        T[j, ..., 1] = ex * math.pi * np.sin(np.pi * X) * np.cos(np.pi * Y)
        T[j, ..., 2] = ee * math.pi * np.cos(np.pi * X) * np.sin(2 * np.pi * Y)
        T[j, ..., 3] = ee * 2 * math.pi * np.sin(np.pi * X) * np.cos(2 * np.pi * Y)
    xs, ys = np.full(3, 0.5), np.array([0.375, 0.5, 0.625])
    kw = dict(dt=dt, Dt=Dt, seed=0, exit_mode=1)
    plain = oracle_mod.interface_mc(P, xs, ys, 4000, **kw)
    exact = oracle_mod.interface_mc(P, xs, ys, 4000, cv_table=T, **kw)
    # what is left is the sub-step discretisation (exits between sub-steps, second-order terms),
    # which shrinks like sqrt(dt): about 7x (xi) and 6x (eta) fewer standard errors at dt = 5e-4
    assert np.all(exact["se_xi"] < plain["se_xi"] / 5), (plain["se_xi"], exact["se_xi"])
    assert np.all(exact["se_eta"] < plain["se_eta"] / 4.5), (plain["se_eta"], exact["se_eta"])
    # the sign and the sqrt(2) scale are pinned: a flipped or a rescaled model does worse
    flipped = oracle_mod.interface_mc(P, xs, ys, 4000, cv_table=-T, **kw)
    assert np.all(flipped["se_xi"] > plain["se_xi"])
    scaled = oracle_mod.interface_mc(P, xs, ys, 4000, cv_table=T / math.sqrt(2), **kw)
    assert np.all(scaled["se_xi"] > 1.5 * exact["se_xi"])
    # and the corrected mean is the closed form up to the method's own bias
    ex, ee = W.heat_exact(xs, ys, Dt)
    assert np.all(np.abs(exact["mean_xi"] - ex) < 2e-3), exact["mean_xi"] - ex


def test_field_gradient_model(oracle_mod):
    # the untrained model: finite-difference gradients of the fields at t_{n-1}
    from oracle import mlp
    n = 65
    X, Y = W.grid(n)
    xi0 = X + 0.02 * np.sin(np.pi * X) * np.sin(np.pi * Y)
    eta0 = Y.copy()
    T = mlp.field_gradient_table(xi0, eta0)
    assert T.shape == (1, n, n, 4)
    np.testing.assert_allclose(T[0, ..., 3], 1.0, atol=1e-12)        # d eta / dy of eta = y
    np.testing.assert_allclose(T[0, ..., 2], 0.0, atol=1e-12)
    P = oracle_mod.Problem(W.w_front(n, 0.1), xi0, eta0)
    xs, ys = W.interface_node_coords(n, n, 2, 2)
    pick = np.arange(0, xs.size, 8)
    kw = dict(dt=1e-4, Dt=1e-2, seed=3)
    a = oracle_mod.interface_mc(P, xs[pick], ys[pick], 2000, **kw)
    b = oracle_mod.interface_mc(P, xs[pick], ys[pick], 2000, cv_table=T, **kw)
    for f, want in (("xi", 3.0), ("eta", 50.0)):
        r = (a["se_" + f] / b["se_" + f]) ** 2
        assert np.median(r) > want, (f, np.median(r))
        assert np.all(np.abs(a["mean_" + f] - b["mean_" + f]) < 4 * np.hypot(a["se_" + f], b["se_" + f]))


def test_pair_evaluated_model_is_unbiased_and_matches_per_step_for_a_static_field(oracle_mod):
    # the model evaluated once per sub-step pair (at X_{2m}, for both increments) is known before
    # both increments, so the estimate stays unbiased; for a model that varies only in space on
    # scales far above a sub-step's spread (the previous fields' gradient) it removes as much
    # variance as the per-sub-step evaluation
    from oracle import mlp
    n = 65
    X, Y = W.grid(n)
    xi0 = X + 0.02 * np.sin(np.pi * X) * np.sin(np.pi * Y)
    eta0 = Y + 0.01 * np.sin(2 * np.pi * X) * np.sin(np.pi * Y)
    T = mlp.field_gradient_table(xi0, eta0)
    P = oracle_mod.Problem(W.w_front(n, 0.1), xi0, eta0)
    xs, ys = W.interface_node_coords(n, n, 2, 2)
    pick = np.arange(0, xs.size, 6)
    kw = dict(dt=1e-4, Dt=1e-2, seed=5, record=True)
    N = 3000
    a = oracle_mod.interface_mc(P, xs[pick], ys[pick], N, **kw)
    b = oracle_mod.interface_mc(P, xs[pick], ys[pick], N, cv_table=T, **kw)
    c = oracle_mod.interface_mc(P, xs[pick], ys[pick], N, cv_table=T, cv_pairs=True, **kw)
    np.testing.assert_array_equal(a["code"], c["code"])
    assert not np.array_equal(b["score_xi"], c["score_xi"])          # the pair evaluation is really used
    for f in ("xi", "eta"):
        rb = np.median((a["se_" + f] / b["se_" + f]) ** 2)
        rc = np.median((a["se_" + f] / c["se_" + f]) ** 2)
        assert rc > 0.9 * rb, (f, rb, rc)
        D = (c["score_" + f] - a["score_" + f]).reshape(pick.size, N)
        z = D.mean(axis=1) / (D.std(axis=1, ddof=1) / math.sqrt(N) + 1e-300)
        assert np.all(np.abs(z) < 4.5), z
    # the bridge test draws per sub-step: no pairs, the flag changes nothing
    d = oracle_mod.interface_mc(P, xs[pick][:3], ys[pick][:3], 500, cv_table=T, cv_pairs=True, exit_mode=1,
                                **{k: v for k, v in kw.items()})
    e = oracle_mod.interface_mc(P, xs[pick][:3], ys[pick][:3], 500, cv_table=T, exit_mode=1, **kw)
    np.testing.assert_array_equal(d["score_xi"], e["score_xi"])
