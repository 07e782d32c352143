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


def test_cell_table_is_the_exact_gradient_of_quadratic_fields():
    # the nodes' differences (central, and second-order one-sided on the edges) are exact on
    # quadratics and the symmetric binomial weights reproduce a linear gradient at the cell
    # centre: every cell whose window stays inside the grid holds the exact gradient at its
    # centre (order 1 has no window past an edge: every cell), and an affine field's constant
    # gradient comes out at every cell for any order
    from oracle import mlp
    nx, ny = 41, 29
    X, Y = W.grid(nx, ny)
    XC, YC = np.meshgrid((np.arange(nx - 1) + 0.5) / (nx - 1), (np.arange(ny - 1) + 0.5) / (ny - 1))
    c = np.random.default_rng(3).normal(size=(2, 6))

    def quad(k, x, y):
        return c[k, 0] * x ** 2 + c[k, 1] * x * y + c[k, 2] * y ** 2 + c[k, 3] * x + c[k, 4] * y + c[k, 5]

    want = np.stack([2 * c[0, 0] * XC + c[0, 1] * YC + c[0, 3], c[0, 1] * XC + 2 * c[0, 2] * YC + c[0, 4],
                     2 * c[1, 0] * XC + c[1, 1] * YC + c[1, 3], c[1, 1] * XC + 2 * c[1, 2] * YC + c[1, 4]], -1)
    for order in (1, 5, 9):
        T = mlp.field_cell_gradient_table(quad(0, X, Y), quad(1, X, Y), order)
        assert T.shape == (1, ny - 1, nx - 1, 4)
        r = (order - 1) // 2
        inner = (slice(r, ny - 1 - r), slice(r, nx - 1 - r))
        np.testing.assert_allclose(T[0][inner], want[inner], rtol=0, atol=1e-11)
        if order > 1:
            assert np.abs(T[0] - want).max() > 1e-3           # the edge windows read the edge nodes
    T1 = mlp.field_cell_gradient_table(quad(0, X, Y), quad(1, X, Y), 1)
    np.testing.assert_allclose(T1[0], want, rtol=0, atol=1e-11)
    for order in (1, 9, 33):
        T = mlp.field_cell_gradient_table(0.3 * X - 1.7 * Y + 0.2, 2.5 * X + 0.4 * Y, order)
        np.testing.assert_allclose(T[0], np.broadcast_to([0.3, -1.7, 2.5, 0.4], T[0].shape), rtol=0, atol=1e-11)
    for order in (0, 2, -1):
        with pytest.raises(ValueError):
            mlp.field_cell_gradient_table(X, Y, order)


def test_cell_model_keeps_the_mean_and_reads_the_cell_of_the_point(oracle_mod):
    # heat problem on 65 x 49 nodes: one value per cell, the exact gradient half-way through the
    # mesh step at the cell's centre
    nx, ny = 65, 49
    X, Y = W.grid(nx, ny)
    xi0, eta0 = np.sin(np.pi * X) * np.sin(np.pi * Y), np.sin(np.pi * X) * np.sin(2 * np.pi * Y)
    P = oracle_mod.Problem(W.w_const(nx, ny), xi0, eta0, np.zeros(oracle_mod.faces_len(nx, ny)))
    dt, Dt = 5e-4, 0.05
    XC, YC = np.meshgrid((np.arange(nx - 1) + 0.5) / (nx - 1), (np.arange(ny - 1) + 0.5) / (ny - 1))
    ex, ee = math.exp(-math.pi ** 2 * Dt), math.exp(-2.5 * math.pi ** 2 * Dt)
    T = np.zeros((1, ny - 1, nx - 1, 4))
    T[0, ..., 0] = ex * math.pi * np.cos(np.pi * XC) * np.sin(np.pi * YC)
    T[0, ..., 1] = ex * math.pi * np.sin(np.pi * XC) * np.cos(np.pi * YC)
    T[0, ..., 2] = ee * math.pi * np.cos(np.pi * XC) * np.sin(2 * np.pi * YC)
    T[0, ..., 3] = ee * 2 * math.pi * np.sin(np.pi * XC) * np.cos(2 * np.pi * YC)
    xs, ys = np.array([0.5, 0.3, 0.7]), np.array([0.375, 0.5, 0.6])
    kw = dict(dt=dt, Dt=Dt, seed=0, record=True)
    N = 4000
    a = oracle_mod.interface_mc(P, xs, ys, N, **kw)
    b = oracle_mod.interface_mc(P, xs, ys, N, cv_table=T, **kw)
    np.testing.assert_array_equal(a["code"], b["code"])
    assert np.all(b["se_xi"] < a["se_xi"] / 3), (a["se_xi"], b["se_xi"])
    assert np.all(b["se_eta"] < a["se_eta"] / 1.5), (a["se_eta"], b["se_eta"])
    for f in ("xi", "eta"):
        D = (b["score_" + f] - a["score_" + f]).reshape(3, N)
        z = D.mean(axis=1) / (D.std(axis=1, ddof=1) / math.sqrt(N))
        assert np.all(np.abs(z) < 4.0), z
    # the rows mirrored (the wrong cell for a point off the middle row): d/dy of the xi model
    # changes sign and the estimate gets worse than without a model
    m = oracle_mod.interface_mc(P, xs, ys, N, cv_table=np.ascontiguousarray(T[:, ::-1]), **kw)
    assert np.all(m["se_xi"] > a["se_xi"]), (a["se_xi"], m["se_xi"])
    # a constant per cell is the constant per node (up to the interpolation's rounding)
    v = np.array([0.7, -0.2, 0.4, 1.1])
    c1 = oracle_mod.interface_mc(P, xs, ys, 500, cv_table=np.broadcast_to(v, (1, ny - 1, nx - 1, 4)), **kw)
    c2 = oracle_mod.interface_mc(P, xs, ys, 500, cv_table=np.broadcast_to(v, (1, ny, nx, 4)), **kw)
    for k in ("steps", "code"):
        np.testing.assert_array_equal(c1[k], c2[k])
    for k in ("score_xi", "score_eta"):
        np.testing.assert_allclose(c1[k], c2[k], rtol=0, atol=1e-13)


def test_smoothed_cell_table_beats_the_node_table_on_noisy_fields(oracle_mod):
    # after mesh steps whose interface values carry Monte Carlo error, the fields' differences
    # are noisy on the grid's scale near the interfaces, where the paths start: the smoothed
    # cell values remove more variance than the node differences themselves
    from oracle import mlp
    n, dt, Dt = 257, 1e-5, 1e-3
    xi, eta = W.identity_fields(n)
    ii, jj = W.interface_nodes(n, n, 8, 8)
    for s in range(3):
        (xi, eta), _ = oracle_mod.dd_step(W.w_ring(n, s * Dt), xi, eta, sub_x=8, sub_y=8, dt=dt, Dt=Dt, n_paths=500,
                                          seed=11, step_index=s, nodes_ij=(ii, jj))
    P = oracle_mod.Problem(W.w_ring(n, 3 * Dt), xi, eta)
    pick = np.random.default_rng(1).choice(ii.size, 48, replace=False)
    xs, ys = ii[pick] / (n - 1), jj[pick] / (n - 1)
    kw = dict(dt=dt, Dt=Dt, seed=5, step_index=3)
    plain = oracle_mod.interface_mc(P, xs, ys, 4000, **kw)
    node = oracle_mod.interface_mc(P, xs, ys, 4000, cv_table=mlp.field_gradient_table(xi, eta), **kw)
    cell = oracle_mod.interface_mc(P, xs, ys, 4000, cv_table=mlp.field_cell_gradient_table(xi, eta, 7), **kw)
    for f in ("xi", "eta"):
        v0, vn, vc = (np.sum(r["se_" + f] ** 2) for r in (plain, node, cell))
        assert v0 / vn > 20, (f, v0 / vn)
        assert vn / vc > 1.5, (f, v0 / vn, v0 / vc)
        z = (cell["mean_" + f] - plain["mean_" + f]) / np.hypot(cell["se_" + f], plain["se_" + f])
        assert np.all(np.abs(z) < 4.5), z
