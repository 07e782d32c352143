"""Pins of the oracle's estimator (Eq. 7b under Euler--Maruyama, Sec. 4)
against closed forms of the relaxed Winslow problem, Eq. (3).

The estimator is biased by the discrete exit test (Sec. 4, "sub-time steps
... to determine sufficiently accurate whether the process has left"); the
closed-form checks therefore use the Brownian-bridge test (reading R7), and
the plain test is pinned by the known sqrt(dt) behaviour of its bias.
"""
import math

import numpy as np
import pytest

import workloads as W


def _zero_faces(oracle_mod, n):
    return np.zeros(oracle_mod.faces_len(n, n))


def test_constant_data_zero_variance(oracle_mod):
    n = 17
    faces = np.full(oracle_mod.faces_len(n, n), 0.625)
    P = oracle_mod.Problem(W.w_smooth_random(n, 1), np.full((n, n), 0.625), np.full((n, n), 0.625), faces)
    xs = np.array([0.5, 0.1, 0.93, 0.0, 1.0])
    ys = np.array([0.5, 0.02, 0.6, 0.3, 1.0])
    for mode in (0, 1):
        r = oracle_mod.interface_mc(P, xs, ys, 300, dt=2e-3, Dt=0.1, exit_mode=mode)
        np.testing.assert_allclose(r["mean_xi"], 0.625, rtol=0, atol=1e-15)
        np.testing.assert_allclose(r["mean_eta"], 0.625, rtol=0, atol=1e-15)
        assert np.all(r["se_xi"] < 1e-14) and np.all(r["se_eta"] < 1e-14)
        # boundary nodes: no path steps; interior nodes: some exits at x = 0.1, 0.02
        assert r["path_steps"][3] == 0 and r["path_steps"][4] == 0
        assert r["n_exit"][1] > 0


def test_heat_equation_closed_form_bridge(oracle_mod):
    # w = 1: Eq. (3) is the heat equation; sin(pi x) sin(pi y) decays by exp(-2 pi^2 t)
    xi0, eta0 = W.heat65_fields()
    P = oracle_mod.Problem(W.w_const(65), xi0, eta0, _zero_faces(oracle_mod, 65))
    xs, ys = W.heat65_nodes()
    r = oracle_mod.interface_mc(P, xs, ys, 20000, dt=1e-3, Dt=0.05, exit_mode=1)
    ex, ee = W.heat_exact(xs, ys, 0.05)
    inner = slice(1, 32)
    # bilinear interpolation of xi0 on 65^2 adds at most ~2e-4 (reading R5)
    zx = np.abs(r["mean_xi"] - ex)[inner] / (r["se_xi"][inner] + 1e-12)
    ze = np.abs(r["mean_eta"] - ee)[inner] / (r["se_eta"][inner] + 1e-12)
    assert np.all(np.abs(r["mean_xi"] - ex)[inner] <= 4 * r["se_xi"][inner] + 3e-4), zx.max()
    assert np.all(np.abs(r["mean_eta"] - ee)[inner] <= 4 * r["se_eta"][inner] + 3e-4), ze.max()
    # and overall the standardised errors look like N(0, 1)
    assert np.mean(zx ** 2) < 2.0 and np.mean(ze ** 2) < 2.0
    # the two ends of the line are boundary nodes: zero data, zero steps
    assert r["mean_xi"][0] == 0 and r["mean_xi"][32] == 0 and r["path_steps"][0] == 0


def test_heat_equation_plain_bias_scales_like_sqrt_dt(oracle_mod):
    # the plain test misses excursions between sub-steps, so it overestimates
    # xi (paths survive too often on a problem with zero boundary data); the
    # bias shrinks like sqrt(dt)
    xi0, eta0 = W.heat65_fields()
    P = oracle_mod.Problem(W.w_const(65), xi0, eta0, _zero_faces(oracle_mod, 65))
    xs = np.full(6, 0.5)
    ys = np.array([0.125, 0.25, 0.375, 0.5, 0.625, 0.75])
    ex, _ = W.heat_exact(xs, ys, 0.05)
    b1 = oracle_mod.interface_mc(P, xs, ys, 40000, dt=1e-3, Dt=0.05, exit_mode=0)["mean_xi"] - ex
    b4 = oracle_mod.interface_mc(P, xs, ys, 40000, dt=2.5e-4, Dt=0.05, exit_mode=0)["mean_xi"] - ex
    assert np.all(b1 > 0.008)
    ratio = b1.mean() / b4.mean()
    assert 1.5 < ratio < 2.7, (b1, b4)


def _survival_1d(x, t, terms=200):
    # u_t = u_xx on (0, 1), u(0) = 1, zero boundary values
    k = 2 * np.arange(terms) + 1
    return float(np.sum(4.0 / (np.pi * k) * np.sin(k * np.pi * x) * np.exp(-(k * np.pi) ** 2 * t)))


def test_survival_probability_bridge(oracle_mod):
    # w = 1, xi0 = 1, zero boundary data: xi(t, x, y) = P(tau > t), a product of 1D series
    n = 33
    P = oracle_mod.Problem(W.w_const(n), np.ones((n, n)), np.ones((n, n)), _zero_faces(oracle_mod, n))
    xs = np.array([0.5, 0.2, 0.1, 0.05, 0.1, 0.3])
    ys = np.array([0.5, 0.5, 0.1, 0.5, 0.9, 0.05])
    t = 0.02
    r = oracle_mod.interface_mc(P, xs, ys, 40000, dt=5e-4, Dt=t, exit_mode=1)
    want = np.array([_survival_1d(x, t) * _survival_1d(y, t) for x, y in zip(xs, ys)])
    assert np.all(np.abs(r["mean_xi"] - want) <= 4 * r["se_xi"] + 1e-3), (r["mean_xi"], want, r["se_xi"])
    # the exit count agrees with the survival probability too
    frac_exit = r["n_exit"] / 40000
    assert np.all(np.abs(frac_exit - (1 - want)) <= 4 * r["se_xi"] + 1e-3)


def test_constant_drift_closed_form(oracle_mod):
    # w = exp(a x): b = (-a, 0). With c = -a, L u = c u_x + u_xx + u_yy has the
    # Dirichlet eigenfunction exp(-c x / 2) sin(pi x) sin(pi y) with eigenvalue
    # -(2 pi^2 + c^2 / 4). A wrong drift sign or scale moves the mean.
    n = 65
    a = 2.0
    X, Y = W.grid(n)
    w = np.exp(a * X).astype(np.float32)
    c = -a
    u0 = np.exp(-c * X / 2) * np.sin(np.pi * X) * np.sin(np.pi * Y)
    P = oracle_mod.Problem(w, u0, u0, _zero_faces(oracle_mod, n))
    xs = np.array([0.25, 0.5, 0.75, 0.5])
    ys = np.array([0.5, 0.5, 0.5, 0.25])
    t = 0.03
    r = oracle_mod.interface_mc(P, xs, ys, 40000, dt=5e-4, Dt=t, exit_mode=1)
    want = np.exp(-c * xs / 2) * np.sin(np.pi * xs) * np.sin(np.pi * ys) * math.exp(-(2 * math.pi ** 2 + c * c / 4) * t)
    assert np.all(np.abs(r["mean_xi"] - want) <= 4 * r["se_xi"] + 1e-3), (r["mean_xi"], want, r["se_xi"])
    flipped = np.exp(c * xs / 2) * np.sin(np.pi * xs) * np.sin(np.pi * ys) * math.exp(-(2 * math.pi ** 2 + c * c / 4) * t)
    assert np.abs(r["mean_xi"] - flipped)[0] > 10 * r["se_xi"][0]


def test_one_dimensional_steady_state(oracle_mod):
    # w = w(x): xi = int_0^x w / int_0^1 w solves Eq. (3) and is stationary;
    # its discrete version is the cumulative trapezoid of w (reading R12)
    n = 65
    X, Y = W.grid(n)
    w = (1.0 + 4.0 * np.exp(-((X - 0.45) / 0.15) ** 2)).astype(np.float32)
    faces = oracle_mod.winslow_faces(w.astype(np.float64))
    seg = oracle_mod.split_faces(faces, n, n)
    xi0 = np.tile(seg[(0, 2)], (n, 1))
    P = oracle_mod.Problem(w, xi0, Y.copy(), faces)
    xs = np.array([0.3, 0.45, 0.5, 0.6, 0.5])
    ys = np.array([0.5, 0.5, 0.3, 0.5, 0.9])
    r = oracle_mod.interface_mc(P, xs, ys, 40000, dt=2.5e-4, Dt=0.01, exit_mode=1)
    want = np.array([oracle_mod.bilinear(xi0, x, y) for x, y in zip(xs, ys)])
    # drift is bilinear between FD nodes: O(h^2) model error, well below 1e-3 here
    assert np.all(np.abs(r["mean_xi"] - want) <= 4 * r["se_xi"] + 1e-3), (r["mean_xi"], want, r["se_xi"])
    assert np.all(np.abs(r["mean_eta"] - ys) <= 4 * r["se_eta"] + 1e-3)


def test_linear_field_reflection_symmetry(oracle_mod):
    # w = 1, xi0 = x and Winslow faces (xi = x on y = 0, 1): on x = 1/2 the law
    # of paths is symmetric under x -> 1 - x, so E = 1/2 for any dt (plain test)
    n = 33
    X, Y = W.grid(n)
    P = oracle_mod.Problem(W.w_const(n), X.copy(), Y.copy())
    xs = np.full(3, 0.5)
    ys = np.array([0.1, 0.5, 0.95])
    r = oracle_mod.interface_mc(P, xs, ys, 40000, dt=1e-3, Dt=0.05, exit_mode=0)
    assert np.all(np.abs(r["mean_xi"] - 0.5) <= 4 * r["se_xi"])
    assert np.all(r["se_xi"] > 0)


def test_record_mode_agrees_with_stats(oracle_mod):
    n = 33
    X, Y = W.grid(n)
    P = oracle_mod.Problem(W.w_smooth_random(n, 5), X.copy(), Y.copy())
    xs = np.array([0.5, 0.05, 0.97])
    ys = np.array([0.5, 0.5, 0.02])
    npaths = np.array([500, 300, 200])
    r = oracle_mod.interface_mc(P, xs, ys, npaths, dt=1e-3, Dt=0.04, exit_mode=0, record=True)
    off = np.concatenate([[0], np.cumsum(npaths)])
    for k in range(3):
        sl = slice(off[k], off[k + 1])
        assert r["mean_xi"][k] == pytest.approx(r["score_xi"][sl].mean(), rel=1e-12)
        assert r["n_exit"][k] == np.sum(r["code"][sl] >= 0)
        assert r["path_steps"][k] == r["steps"][sl].sum()
        # exited paths end on the boundary, survivors run all K = 40 sub-steps
        ex = r["code"][sl] >= 0
        xe, ye = r["x_end"][sl][ex], r["y_end"][sl][ex]
        assert np.all((xe == 0) | (xe == 1) | (ye == 0) | (ye == 1))
        assert np.all(r["steps"][sl][~ex] == 40)


def test_path_increments_have_the_brownian_variance(oracle_mod):
    # w = 1, far from the boundary over a short step: X(Dt) - X(0) = sqrt(2) W(Dt),
    # variance 2 Dt per coordinate, the two coordinates uncorrelated. Reusing or
    # correlating the normals of successive sub-steps changes this.
    n = 17
    X, Y = W.grid(n)
    P = oracle_mod.Problem(W.w_const(n), X.copy(), Y.copy())
    N = 40000
    for mode in (0, 1):
        r = oracle_mod.interface_mc(P, [0.5], [0.5], N, dt=2e-4, Dt=4e-3, exit_mode=mode, record=True)
        assert r["n_exit"][0] == 0
        dx = r["x_end"] - 0.5
        dy = r["y_end"] - 0.5
        for d in (dx, dy):
            assert abs(d.mean()) < 4 * math.sqrt(8e-3 / N)
            assert d.var() == pytest.approx(8e-3, rel=4 * math.sqrt(2 / N))
        assert abs(np.corrcoef(dx, dy)[0, 1]) < 4 / math.sqrt(N)


def test_oracle_regression_fixture(oracle_mod):
    # the stored outputs were written by tests/golden/make_golden.py from this oracle
    import json
    import os
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
    import make_golden
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_regression.json")) as f:
        stored = json.load(f)
    fresh = {"heat65_plain": make_golden.heat65_case(0), "heat65_bridge": make_golden.heat65_case(1),
             "front65_plain": make_golden.front_case(), "front65_cell_cv": make_golden.front_cell_cv_case()}
    for case, got in fresh.items():
        for key, val in got.items():
            np.testing.assert_allclose(np.asarray(val, float), np.asarray(stored[case][key], float),
                                       rtol=1e-9, atol=1e-12, err_msg=f"{case}/{key}")


def test_exponential_time_stepping_heat_closed_form(oracle_mod):
    # exit_mode 2 (exponential sub-step lengths, bridge test over each): for Brownian motion the exit
    # detection is exact, so even five sub-steps on average per mesh step give the closed form
    xi0, eta0 = W.heat65_fields()
    P = oracle_mod.Problem(W.w_const(65), xi0, eta0, _zero_faces(oracle_mod, 65))
    xs, ys = W.heat65_nodes()
    xs, ys = xs[1:32:3], ys[1:32:3]
    r = oracle_mod.interface_mc(P, xs, ys, 40000, dt=1e-2, Dt=0.05, exit_mode=2)
    ex, ee = W.heat_exact(xs, ys, 0.05)
    assert np.all(np.abs(r["mean_xi"] - ex) <= 4 * r["se_xi"] + 3e-4), np.abs(r["mean_xi"] - ex) / r["se_xi"]
    assert np.all(np.abs(r["mean_eta"] - ee) <= 4 * r["se_eta"] + 3e-4)
    # the plain fixed-step test at the same dt is off by far more
    p = oracle_mod.interface_mc(P, xs, ys, 40000, dt=1e-2, Dt=0.05, exit_mode=0)
    assert np.sqrt(np.mean((p["mean_xi"] - ex) ** 2)) > 20 * np.sqrt(np.mean((r["mean_xi"] - ex) ** 2))


def test_exponential_time_stepping_counts_poisson_steps(oracle_mod):
    # far from the boundary every path survives: the sub-step count is the number of exponential
    # arrivals in the mesh step (Poisson with mean K) plus the cut last sub-step, mean K + 1
    n = 33
    P = oracle_mod.Problem(W.w_const(n), *W.identity_fields(n))
    K, N = 20, 20000
    r = oracle_mod.interface_mc(P, [0.5], [0.5], N, dt=1e-5, Dt=K * 1e-5, exit_mode=2, record=True)
    assert r["n_exit"][0] == 0
    steps = r["steps"].astype(np.float64)
    assert abs(steps.mean() - (K + 1)) < 4 * math.sqrt(K / N), steps.mean()
    assert abs(steps.var() - K) < 0.1 * K, steps.var()   # Poisson: variance = mean - 1 here
    # a linear field is preserved exactly whatever the step lengths (zero drift, symmetric increments)
    assert abs(r["mean_xi"][0] - 0.5) < 4 * r["se_xi"][0] + 1e-12


def test_path_margin_follows_the_path(oracle_mod):
    """The margin over the first sub-step of a w = 1 path is the distance of
    X_1 = X_0 + sqrt(2 dt) Z to the nearest boundary line, Z the first normal
    pair of the path's Philox block; over the whole step it never exceeds that."""
    n, dt, Dt, seed = 33, 1e-3, 2e-2, 3
    P = oracle_mod.Problem(W.w_const(n), *W.identity_fields(n))
    x0, y0, node, paths = 0.1, 0.93, 7, np.arange(40)
    ctrs = np.stack([paths, np.full(40, node), np.zeros(40), np.zeros(40)], axis=1)
    _, z = oracle_mod.draw(seed, ctrs)
    x1 = x0 + math.sqrt(2 * dt) * z[:, 0]
    y1 = y0 + math.sqrt(2 * dt) * z[:, 1]
    want = np.minimum(np.minimum(np.abs(x1), np.abs(1 - x1)), np.minimum(np.abs(y1), np.abs(1 - y1)))
    one = oracle_mod.path_margins(P, np.full(40, x0), np.full(40, y0), np.full(40, node), paths, np.ones(40),
                                  dt=dt, Dt=Dt, seed=seed)
    np.testing.assert_allclose(one, want, rtol=1e-12, atol=1e-15)
    r = oracle_mod.interface_mc(P, [x0], [y0], 40, dt=dt, Dt=Dt, seed=seed, node_ids=[node], record=True)
    full = oracle_mod.path_margins(P, np.full(40, x0), np.full(40, y0), np.full(40, node), paths, r["steps"],
                                   dt=dt, Dt=Dt, seed=seed)
    assert np.all(full <= one)
