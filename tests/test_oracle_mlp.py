"""Pins of the oracle's control-variate network: backpropagation and forward-mode
derivatives against central finite differences, Adam's first steps in closed
form, the feature fields against the drift's own finite differences, and the
training data against the heat problem's closed form."""
import math

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def mlp(oracle_mod):
    from oracle import mlp as m
    return m


def _rand_theta(mlp, seed, scale=0.6):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, size=mlp.P)


def test_layout_and_hand_computed_forward(mlp):
    assert mlp.P == 4609
    # one live unit in each layer: g = w3_0 tanh(W2_00 tanh(W1_0 . z + b1_0) + b2_0) + b3
    th = np.zeros(mlp.P)
    p = mlp.unpack(th)
    p["W1"][0] = [0.3, -0.2, 0.5, 0.1, -0.4]
    p["b1"][0] = 0.05
    p["W2"][0, 0] = 1.7
    p["b2"][0] = -0.3
    p["w3"][0] = 2.5
    p["b3"][0] = 0.125
    z = np.array([0.9, -1.1, 0.2, 0.4, 1.3])
    want = 2.5 * math.tanh(1.7 * math.tanh(0.3 * 0.9 + 0.2 * 1.1 + 0.1 + 0.04 - 0.52 + 0.05) - 0.3) + 0.125
    got, _ = mlp.forward(th, z[None, :])
    assert abs(got[0] - want) < 1e-15
    # every other unit is dead: tanh(b2_j) w3_j with w3_j = 0
    p["w3"][1:] = 0.0
    assert abs(mlp.forward(th, z[None, :])[0][0] - want) < 1e-15


def test_backprop_matches_central_differences(mlp):
    rng = np.random.default_rng(1)
    th = _rand_theta(mlp, 2)
    Z = rng.normal(size=(37, 5))
    Y = rng.normal(size=37)
    L, g = mlp.loss_and_grad(th, Z, Y)
    idx = np.concatenate([rng.choice(mlp.P, 300, replace=False), [mlp.P - 1, 0, 320, 383, 4480]])
    h = 1e-6
    for k in idx:
        e = np.zeros(mlp.P)
        e[k] = h
        fd = (mlp.loss_and_grad(th + e, Z, Y)[0] - mlp.loss_and_grad(th - e, Z, Y)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])), (k, fd, g[k])
    # the loss is the mean squared error of forward()
    out, _ = mlp.forward(th, Z)
    assert abs(L - np.mean((out - Y) ** 2)) < 1e-14


def test_forward_mode_matches_central_differences(mlp):
    rng = np.random.default_rng(3)
    th = _rand_theta(mlp, 4)
    Z = rng.normal(size=(20, 5))
    dx = rng.normal(size=(20, 5))
    dy = rng.normal(size=(20, 5))
    g, gx, gy = mlp.input_grad(th, Z, dx, dy)
    h = 1e-6
    fx = (mlp.forward(th, Z + h * dx)[0] - mlp.forward(th, Z - h * dx)[0]) / (2 * h)
    fy = (mlp.forward(th, Z + h * dy)[0] - mlp.forward(th, Z - h * dy)[0]) / (2 * h)
    np.testing.assert_allclose(gx, fx, rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose(gy, fy, rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose(g, mlp.forward(th, Z)[0], rtol=0, atol=1e-15)


def test_adam_first_steps_in_closed_form(mlp):
    rng = np.random.default_rng(5)
    th = rng.normal(size=50)
    g1 = rng.normal(size=50)
    g1[0] = 0.0
    lr = 1e-3
    m = v = np.zeros(50)
    t1, m, v = mlp.adam_update(th, m, v, g1, 1, lr)
    # m-hat = g, v-hat = g^2: each weight moves by lr g / (|g| + eps)
    np.testing.assert_allclose(t1, th - lr * g1 / (np.abs(g1) + 1e-8), rtol=0, atol=1e-15)
    assert t1[0] == th[0]
    g2 = rng.normal(size=50)
    t2, _, _ = mlp.adam_update(t1, m, v, g2, 2, lr)
    mh = (0.9 * 0.1 * g1 + 0.1 * g2) / (1 - 0.81)
    vh = (0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2) / (1 - 0.999 ** 2)
    np.testing.assert_allclose(t2, t1 - lr * mh / (np.sqrt(vh) + 1e-8), rtol=0, atol=1e-15)


def test_learning_rate_schedule(mlp):
    assert mlp.lr_at(0, 100, 3e-3) == 3e-3
    assert abs(mlp.lr_at(50, 100, 3e-3) - 1.5e-3) < 1e-18
    assert abs(mlp.lr_at(100, 100, 3e-3)) < 1e-18


def test_init_weights(mlp):
    a = mlp.init_params(7)
    b = mlp.init_params(7)
    c = mlp.init_params(8)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
    np.testing.assert_array_equal(a, a.astype(np.float32).astype(np.float64))
    for f in range(2):
        p = mlp.unpack(a[f])
        for name, lim in (("W1", math.sqrt(6 / 69)), ("W2", math.sqrt(6 / 128)), ("w3", math.sqrt(6 / 65))):
            x = p[name].ravel()
            assert np.all(np.abs(x) < lim)
            assert abs(x.mean()) < 4 * lim / math.sqrt(3 * x.size)
            # sample variance of n uniforms on [-L, L]: L^2 / 3 with standard deviation L^2 sqrt(4 / (45 n))
            assert abs(x.var() - lim ** 2 / 3) < 4 * lim ** 2 * math.sqrt(4 / (45 * x.size))
        for name in ("b1", "b2", "b3"):
            assert np.all(p[name] == 0)
    assert not np.array_equal(a[0], a[1])


def test_feature_fields(mlp, oracle_mod):
    # the finite differences are exact on quadratics, and agree with the drift's own (C) code
    n = 33
    X, Y = W.grid(n)
    q = 1.0 + 0.5 * X * X - 0.25 * X * Y + 0.75 * Y * Y
    gx, gy = mlp.fd_grad(q)
    np.testing.assert_allclose(gx, X - 0.25 * Y, atol=1e-12)
    np.testing.assert_allclose(gy, -0.25 * X + 1.5 * Y, atol=1e-12)
    w = W.w_front(n, 0.2)
    bx, by = oracle_mod.drift_field(w)
    nf = mlp.node_features(w)
    np.testing.assert_allclose(nf["wx"], -w * bx, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(nf["wy"], -w * by, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(nf["r"], np.hypot(bx, by), rtol=1e-12, atol=1e-12)
    # bilinear interpolation of the features is exact at the nodes and linear along edges
    F = mlp.features(nf, X.ravel(), Y.ravel(), 0.5)
    np.testing.assert_allclose(F[:, 3], w.ravel(), rtol=1e-14)
    np.testing.assert_allclose(F[:, 4], nf["r"].ravel(), rtol=1e-14)
    mid = mlp.features(nf, [0.5 / (n - 1)], [0.0], 1.0)
    assert abs(mid[0, 3] - 0.5 * (w[0, 0] + w[0, 1])) < 1e-14


def test_standardisation(mlp):
    rng = np.random.default_rng(9)
    F = np.column_stack([rng.uniform(size=1000), rng.normal(3, 2, 1000), np.full(1000, 0.7),
                         rng.exponential(size=1000), np.full(1000, 2.0)])
    mu, s = mlp.standardise(F)
    Z = mlp.normalise(F, mu, s)
    np.testing.assert_allclose(Z[:, [0, 1, 3]].mean(axis=0), 0, atol=1e-12)
    np.testing.assert_allclose(Z[:, [0, 1, 3]].std(axis=0), 1, atol=1e-12)
    assert s[2] == 0 and s[4] == 0
    assert np.all(Z[:, [2, 4]] == 0)


def test_slices(mlp):
    assert mlp.slice_bounds(50, 50) == list(range(51))
    np.testing.assert_allclose(mlp.slice_time_fracs(50, 50), [(50 - j) / 50 for j in range(50)])
    assert mlp.slice_bounds(10, 3) == [0, 4, 7, 10]
    np.testing.assert_allclose(mlp.slice_time_fracs(10, 3), [(10 - 1.5) / 10, (10 - 5) / 10, (10 - 8) / 10])


def test_tabulated_gradient_of_a_known_network(mlp):
    # with w = 1 the table is d g / dx = s_x dg/dz_x: compare with finite differences in x itself
    n = 17
    th = np.stack([_rand_theta(mlp, 11, 0.4), _rand_theta(mlp, 12, 0.4)])
    mu = np.array([0.5, 0.5, 0.5, 1.0, 0.0])
    s = np.array([3.0, 2.0, 1.5, 0.0, 0.0])
    T = mlp.tabulate(th, mu, s, np.ones((n, n)), 10, 3)
    X, Y = W.grid(n)
    h = 1e-6
    for q, tf in enumerate(mlp.slice_time_fracs(10, 3)):
        def g(f, x, y):
            F = np.stack([x.ravel(), y.ravel(), np.full(x.size, tf), np.ones(x.size), np.zeros(x.size)], axis=1)
            return mlp.forward(th[f], mlp.normalise(F, mu, s))[0].reshape(x.shape)
        for f in range(2):
            np.testing.assert_allclose(T[q, ..., 2 * f], (g(f, X + h, Y) - g(f, X - h, Y)) / (2 * h), atol=1e-7)
            np.testing.assert_allclose(T[q, ..., 2 * f + 1], (g(f, X, Y + h) - g(f, X, Y - h)) / (2 * h), atol=1e-7)


def test_training_samples_follow_the_heat_solution(mlp, oracle_mod):
    # w = 1 heat problem: E[Y | horizon k] over uniform starts = exp(-2 pi^2 k dt) (2/pi)^2 for xi
    xi0, eta0 = W.heat65_fields()
    faces = np.zeros(oracle_mod.faces_len(65, 65))
    P = oracle_mod.Problem(W.w_const(65), xi0, eta0, faces)
    dt, Dt, M = 1e-3, 0.01, 20000
    F, Y = mlp.training_samples(P, per_horizon=M, dt=dt, Dt=Dt, seed=3, exit_mode=1)
    K = 10
    assert F.shape == (M * K, 5) and Y.shape == (M * K, 2)
    for k in range(1, K + 1):
        rows = np.arange(M) * K + (k - 1)
        np.testing.assert_array_equal(F[rows, 2], k / K)
        want = math.exp(-2 * math.pi ** 2 * k * dt) * (2 / math.pi) ** 2
        se = Y[rows, 0].std() / math.sqrt(M)
        assert abs(Y[rows, 0].mean() - want) < 4 * se + 1e-3, (k, Y[rows, 0].mean(), want)
        assert abs(Y[rows, 1].mean()) < 4 * Y[rows, 1].std() / math.sqrt(M) + 1e-3
    assert np.all((F[:, :2] > 0) & (F[:, :2] < 1))
    # one row, recomputed as a single-path estimate at its own start
    k, m = 7, 123
    word = (k - 1) * M + m
    xs, ys = mlp.sample_starts(3, [word])
    r = oracle_mod.interface_mc(P, xs, ys, 1, dt=dt, Dt=k * dt, seed=3, exit_mode=1,
                                step_index=mlp.SAMPLE_STEP_WORD, node_ids=np.array([word], np.uint32))
    row = m * K + k - 1
    assert F[row, 0] == xs[0] and F[row, 1] == ys[0]
    assert Y[row, 0] == r["mean_xi"][0] and Y[row, 1] == r["mean_eta"][0]


def test_learned_model_reduces_the_variance(mlp, oracle_mod):
    # a short training run on the method's own samples already cuts the variance severalfold
    n, dt, Dt, K = 65, 1e-3, 0.05, 50
    xi0, eta0 = W.heat65_fields()
    P = oracle_mod.Problem(W.w_const(n), xi0, eta0, np.zeros(oracle_mod.faces_len(n, n)))
    F, Y = mlp.training_samples(P, per_horizon=4000, dt=dt, Dt=Dt, seed=1)
    mu, s = mlp.standardise(F)
    Z = mlp.normalise(F, mu, s)
    th0 = mlp.init_params(7)
    thetas = []
    for f in range(2):
        th, losses = mlp.train(th0[f], Z, Y[:, f], epochs=5, batch=4096, lr0=3e-3)
        assert np.mean(losses[-20:]) < 0.8 * losses[0]   # most of what is left is the scores' own noise
        thetas.append(th)
    T = mlp.tabulate(thetas, mu, s, P.w, K, K)
    xs, ys = W.heat65_nodes()
    kw = dict(dt=dt, Dt=Dt, seed=0)
    plain = oracle_mod.interface_mc(P, xs, ys, 2000, **kw)
    cv = oracle_mod.interface_mc(P, xs, ys, 2000, cv_table=T, **kw)
    inner = slice(1, 32)
    for f in ("xi", "eta"):
        ratio = (plain["se_" + f][inner] / cv["se_" + f][inner]) ** 2
        assert np.median(ratio) > 3, (f, np.median(ratio))
        d = np.abs(cv["mean_" + f] - plain["mean_" + f])[inner]
        assert np.all(d < 4 * np.hypot(cv["se_" + f], plain["se_" + f])[inner] + 1e-12)
