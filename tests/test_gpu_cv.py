"""The control-variate path on the GPU against the oracle's control-variate estimator.

Y_cv = Y - sum_{j < kappa} G(s_j, X_j) . sqrt(2) dW_j, the model G given as a
node table in space and piecewise constant in time. The same Philox streams
drive both sides, so the records must agree path by path (the paths are not
moved by the model; only the score changes).
"""
import math

import numpy as np
import pytest

import workloads as W
from tests import _parity as PT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sdd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1402_0266_gb300 import build
    build.build()
    import paper_1402_0266_gb300 as m
    return m


def _np(d):
    return {k: v.cpu().numpy() for k, v in d.items()}


def _ctx(sdd, w, xi0, eta0, sub=2, faces=None):
    import torch
    ny, nx = w.shape
    ctx = sdd.sdd_init(nx, ny, sub, sub, w=torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda(),
                       xi0=torch.from_numpy(np.ascontiguousarray(xi0)).cuda(),
                       eta0=torch.from_numpy(np.ascontiguousarray(eta0)).cuda())
    if faces is not None:
        sdd.sdd_set_boundary(ctx, torch.from_numpy(np.ascontiguousarray(faces, np.float64)).cuda())
    return ctx


def _h(T):
    """The model the GPU uses: the table's node values rounded to half precision."""
    return np.asarray(T, dtype=np.float16).astype(np.float64)


def _f(T):
    """Cell values as the GPU keeps them: single precision."""
    return np.asarray(T, dtype=np.float32).astype(np.float64)


def _set_table(sdd, ctx, T):
    import torch
    sdd.sdd_cv_set_table(ctx, torch.from_numpy(np.ascontiguousarray(T, np.float64)).cuda())


def _smooth_table(n, S):
    X, Y = W.grid(n)
    T = np.zeros((S, n, n, 4))
    for q in range(S):
        T[q, ..., 0] = 2.0 * np.sin(3 * X + q) * np.cos(2 * Y)
        T[q, ..., 1] = 1.5 + np.cos(5 * X * Y)
        T[q, ..., 2] = -3.0 * X * Y + 0.3 * q
        T[q, ..., 3] = np.sin(4 * Y - X)
    return T


def _heat_table(n, dt, Dt):
    # grad of exp(-2 pi^2 s) sin(pi x) sin(pi y) and exp(-5 pi^2 s) sin(pi x) sin(2 pi y),
    # s = Dt - j dt the time left at sub-step j; one slice per sub-step
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
    return T


# odd K in the paired kernel (the last pair takes one sub-step), even K, the bridge kernel;
# slice counts that split K unevenly, and one slice per sub-step
CASES = [(0, 1e-3, 0.049, 5), (0, 1e-3, 0.05, 50), (1, 1e-3, 0.05, 7), (0, 5e-4, 0.02, 3)]


@pytest.mark.parametrize("exit_mode,dt,Dt,S", CASES)
def test_cv_records_match_oracle(sdd, oracle_mod, exit_mode, dt, Dt, S):
    n = 65
    w = W.w_front(n, 0.1)
    xi0, eta0 = W.identity_fields(n)
    ctx = _ctx(sdd, w, xi0, eta0)
    T = _smooth_table(n, S)
    _set_table(sdd, ctx, T)
    sdd.sdd_cv_enable(ctx, True)
    xs, ys = W.interface_node_coords(n, n, 2, 2)
    pick = np.arange(0, xs.size, 9)
    xs = np.concatenate([xs[pick], [0.0, 0.013]])
    ys = np.concatenate([ys[pick], [0.4, 0.77]])
    npaths = np.full(xs.size, 700)
    npaths[::3] = 41
    kw = dict(dt=dt, Dt=Dt, seed=5, step_index=2, exit_mode=exit_mode)
    g = _np(sdd.sdd_interface_mc_record(ctx, xs, ys, npaths, **kw))
    P = oracle_mod.Problem(w, xi0, eta0)
    o = oracle_mod.interface_mc(P, xs, ys, npaths, record=True, cv_table=_h(T), **kw)
    plain = oracle_mod.interface_mc(P, xs, ys, npaths, record=True, **kw)
    # the table really enters the scores
    assert np.abs(o["score_xi"] - plain["score_xi"]).max() > 1e-2
    same, rep = PT.assert_records(g, o)
    offsets = np.concatenate([[0], np.cumsum(npaths)])
    PT.assert_nodes(g, o, npaths, same, offsets)


def test_cv_zero_table_gives_the_plain_estimate(sdd):
    n = 65
    w = W.w_ring(n, 0.1)
    xi0, eta0 = W.identity_fields(n)
    ctx = _ctx(sdd, w, xi0, eta0)
    xs, ys = W.interface_node_coords(n, n, 2, 2)
    npaths = np.full(xs.size, 500)
    kw = dict(dt=1e-3, Dt=0.03, seed=3)
    plain = _np(sdd.sdd_interface_mc(ctx, xs, ys, npaths, **kw))
    _set_table(sdd, ctx, np.zeros((4, n, n, 4)))
    sdd.sdd_cv_enable(ctx, True)
    cv = _np(sdd.sdd_interface_mc(ctx, xs, ys, npaths, **kw))
    for k in ("mean_xi", "mean_eta", "se_xi", "se_eta"):
        np.testing.assert_allclose(cv[k], plain[k], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(cv["n_exit"], plain["n_exit"])
    np.testing.assert_array_equal(cv["path_steps"], plain["path_steps"])
    sdd.sdd_cv_enable(ctx, False)
    again = _np(sdd.sdd_interface_mc(ctx, xs, ys, npaths, **kw))
    np.testing.assert_array_equal(again["mean_xi"], plain["mean_xi"])


def test_cv_exact_gradient_shrinks_the_error_on_gpu(sdd, oracle_mod):
    n, dt, Dt = 65, 5e-4, 0.05
    xi0, eta0 = W.heat65_fields()
    faces = np.zeros(oracle_mod.faces_len(n, n))
    ctx = _ctx(sdd, W.w_const(n), xi0, eta0, faces=faces)
    xs, ys = W.heat65_nodes()
    npaths = np.full(xs.size, 4000)
    kw = dict(dt=dt, Dt=Dt, seed=0, exit_mode=1)
    plain = _np(sdd.sdd_interface_mc(ctx, xs, ys, npaths, **kw))
    T = _heat_table(n, dt, Dt)
    _set_table(sdd, ctx, T)
    sdd.sdd_cv_enable(ctx, True)
    cv = _np(sdd.sdd_interface_mc(ctx, xs, ys, npaths, **kw))
    inner = (xs > 0) & (xs < 1) & (ys > 0) & (ys < 1)
    # what is left is the sub-step discretisation, larger near the boundary where more paths exit
    for f in ("xi", "eta"):
        ratio = plain["se_" + f][inner] / cv["se_" + f][inner]
        assert np.all(ratio > 3.5), (f, ratio.min())
        assert np.median(ratio) > 5, (f, np.median(ratio))
    ex, ee = W.heat_exact(xs, ys, Dt)
    # within the (now small) statistical error plus the sub-step bias of the method
    assert np.all(np.abs(cv["mean_xi"] - ex)[inner] < 4 * cv["se_xi"][inner] + 3e-4)
    assert np.all(np.abs(cv["mean_eta"] - ee)[inner] < 4 * cv["se_eta"][inner] + 3e-4)
    # and the same numbers as the oracle's control-variate estimator on a few nodes
    sel = np.flatnonzero(inner)[::8]
    P = oracle_mod.Problem(W.w_const(n), xi0, eta0, faces)
    o = oracle_mod.interface_mc(P, xs[sel], ys[sel], npaths[sel], cv_table=_h(T), node_ids=sel.astype(np.uint32),
                                **kw)
    for f in ("xi", "eta"):
        d = np.abs(cv["mean_" + f][sel] - o["mean_" + f])
        assert np.all(d <= 3 * o["se_" + f] + 1e-4), (f, d)
        np.testing.assert_allclose(cv["se_" + f][sel], o["se_" + f], rtol=0.05)


def test_cv_mesh_step_matches_oracle(sdd, oracle_mod):
    n, sub, dt, Dt, paths = 33, 2, 1e-4, 1e-2, 1500
    w = W.w_front(n, 0.0)
    xi0, eta0 = W.identity_fields(n)
    ctx = _ctx(sdd, w, xi0, eta0, sub)
    T = _smooth_table(n, 10)
    _set_table(sdd, ctx, T)
    sdd.sdd_cv_enable(ctx, True)
    sdd.sdd_step(ctx, dt=dt, Dt=Dt, seed=9, paths_per_node=paths, rtol=1e-13, max_iter=50000)
    sdd.sdd_sync(ctx)
    g = _np(sdd.sdd_last_interface_stats(ctx))
    ii, jj = W.interface_nodes(n, n, sub, sub)
    new, o = oracle_mod.dd_step(w, xi0, eta0, sub_x=sub, sub_y=sub, dt=dt, Dt=Dt, n_paths=paths, seed=9,
                                step_index=0, nodes_ij=(ii, jj), cv_table=_h(T))
    for f in ("xi", "eta"):
        d = np.abs(g["mean_" + f] - o["mean_" + f])
        assert np.all(d <= 3 * o["se_" + f] + 1e-4), (f, d.max())
        assert np.median(d) <= 1e-5
    gx, ge = (a.cpu().numpy() for a in sdd.sdd_get_fields(ctx))
    iface_gap = max(np.abs(g["mean_xi"] - o["mean_xi"]).max(), np.abs(g["mean_eta"] - o["mean_eta"]).max())
    assert max(np.abs(gx - new[0]).max(), np.abs(ge - new[1]).max()) <= iface_gap + 1e-9


def test_cv_rejections(sdd):
    import torch
    n = 17
    w = np.ones((n, n))
    xi0, eta0 = W.identity_fields(n)
    ctx = _ctx(sdd, w, xi0, eta0)
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_cv_enable(ctx, True)              # no table yet
    assert e.value.status == sdd.SDD_EINVAL
    for S in (0, 129):
        with pytest.raises((sdd.SddError, ValueError)):
            sdd.sdd_cv_set_table(ctx, torch.zeros((S, n, n, 4), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        sdd.sdd_cv_set_table(ctx, torch.zeros((2, n, n, 3), dtype=torch.float64, device="cuda"))
    _set_table(sdd, ctx, np.zeros((20, n, n, 4)))
    sdd.sdd_cv_enable(ctx, True)
    with pytest.raises(sdd.SddError) as e:        # 20 slices, 10 sub-steps
        sdd.sdd_interface_mc(ctx, [0.5], [0.5], [10], dt=1e-3, Dt=1e-2)
    assert e.value.status == sdd.SDD_EINVAL


def test_field_gradient_mode_matches_oracle(sdd, oracle_mod):
    from oracle import mlp
    n = 65
    w = W.w_front(n, 0.1)
    X, Y = W.grid(n)
    xi0 = X + 0.02 * np.sin(np.pi * X) * np.sin(np.pi * Y)
    eta0 = Y.copy()
    ctx = _ctx(sdd, w, xi0, eta0)
    sdd.sdd_cv_enable(ctx, sdd.SDD_CV_FIELDS)
    assert sdd.sdd_cv_fields_order(ctx) == 1          # a 65-node grid: no smoothing by default
    xs, ys = W.interface_node_coords(n, n, 2, 2)
    pick = np.arange(0, xs.size, 5)
    xs, ys = xs[pick], ys[pick]
    npaths = np.full(xs.size, 600)
    T = mlp.field_gradient_table(xi0, eta0)
    for order, mode in ((0, 0), (9, 0), (9, 1)):
        sdd.sdd_cv_set_fields_order(ctx, order)
        o_ = sdd.sdd_cv_fields_order(ctx)
        assert o_ == (order or 1)
        kw = dict(dt=1e-4, Dt=1e-2, seed=6, exit_mode=mode)
        g = _np(sdd.sdd_interface_mc_record(ctx, xs, ys, npaths, **kw))
        np.testing.assert_allclose(sdd.sdd_cv_get_table(ctx, 1).cpu().numpy(), T, rtol=1e-12, atol=1e-9)
        C = mlp.field_cell_gradient_table(xi0, eta0, o_)
        np.testing.assert_allclose(sdd.sdd_cv_get_cells(ctx).cpu().numpy(), C[0], rtol=0, atol=2e-6)
        # the model at every sub-step: the value of the cell the path is in
        o = oracle_mod.interface_mc(oracle_mod.Problem(w, xi0, eta0), xs, ys, npaths, record=True, cv_table=_f(C),
                                    **kw)
        same, rep = PT.assert_records(g, o)
        PT.assert_nodes(g, o, npaths, same, np.concatenate([[0], np.cumsum(npaths)]))
        if (order, mode) == (0, 0):
            g_cells = g
    for bad in (2, -1, 257):
        with pytest.raises(sdd.SddError):
            sdd.sdd_cv_set_fields_order(ctx, bad)
    kw = dict(dt=1e-4, Dt=1e-2, seed=6, exit_mode=0)
    # and a table set by hand is evaluated at every sub-step
    _set_table(sdd, ctx, T)
    sdd.sdd_cv_enable(ctx, sdd.SDD_CV_TABLE)
    g1 = _np(sdd.sdd_interface_mc_record(ctx, xs, ys, npaths, **kw))
    o1 = oracle_mod.interface_mc(oracle_mod.Problem(w, xi0, eta0), xs, ys, npaths, record=True, cv_table=_h(T), **kw)
    same1, _ = PT.assert_records(g1, o1)
    PT.assert_nodes(g1, o1, npaths, same1, np.concatenate([[0], np.cumsum(npaths)]))
    assert not np.array_equal(g1["score_xi"], g_cells["score_xi"])


def test_model_mode_tabulates_before_every_estimate(sdd, oracle_mod):
    # SDD_CV_MODEL rebuilds the table from the context's current w: the same numbers as
    # tabulating by hand and using the table, before and after w changes
    n = 65
    xi0, eta0 = W.identity_fields(n)
    ctx = _ctx(sdd, W.w_front(n, 0.0), xi0, eta0)
    info = sdd.sdd_cv_train(ctx, per_horizon=400, dt=1e-3, Dt=1e-2, seed=2, epochs=2, batch=1024, slices=4)
    theta, norm = sdd.sdd_cv_get_model(ctx)
    xs, ys = W.interface_node_coords(n, n, 2, 2)
    npaths = np.full(xs.size, 300)
    kw = dict(dt=1e-3, Dt=1e-2, seed=8)
    import torch
    for t in (0.0, 0.3):
        sdd.sdd_set_w(ctx, torch.from_numpy(W.w_front(n, t)).cuda())
        sdd.sdd_cv_enable(ctx, sdd.SDD_CV_MODEL)
        a = _np(sdd.sdd_interface_mc(ctx, xs, ys, npaths, **kw))
        sdd.sdd_cv_tabulate(ctx, theta, norm, 4, dt=1e-3, Dt=1e-2)
        sdd.sdd_cv_enable(ctx, sdd.SDD_CV_TABLE)
        b = _np(sdd.sdd_interface_mc(ctx, xs, ys, npaths, **kw))
        for k in ("mean_xi", "mean_eta", "se_xi", "se_eta"):
            np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("mode", ["fields", "model"])
def test_mesh_steps_with_control_variate_match_oracle(sdd, oracle_mod, mode):
    # the GPU's trajectory and the oracle's from the same start, each on its own fields and with
    # its own model table: the field gradient from its own fields, or a seeded network (weights
    # and standardisation of the oracle's training samples, given to both) tabulated by each side
    # from each step's w. The two sides' control-variate sums differ (other fields, BF16 tensor
    # cores against FP64) by a term of mean zero, so the node means may differ by 3 (SE_gpu +
    # SE_oracle), a bound on three standard deviations of the difference of the two correlated
    # estimates, plus the previous fields' gap
    from oracle import mlp
    import torch
    n, sub, dt, Dt, paths, S = 33, 2, 1e-4, 1e-2, 1500, 4
    K = int(round(Dt / dt))
    xi0, eta0 = W.identity_fields(n)
    ctx = _ctx(sdd, W.w_front(n, 0.0), xi0, eta0, sub)
    if mode == "model":
        P_ = oracle_mod.Problem(W.w_front(n, 0.0), xi0, eta0)
        F, _ = mlp.training_samples(P_, per_horizon=20, dt=dt, Dt=Dt, seed=2)
        mu, sd = mlp.standardise(F)
        th = mlp.init_params(3) + 0.2 * np.random.default_rng(3).normal(size=(2, mlp.P))
        th = th.astype(np.float32).astype(np.float64)
        block = np.zeros(2 * sdd.MLP_STRIDE, np.float32)
        block[:mlp.P], block[sdd.MLP_STRIDE:sdd.MLP_STRIDE + mlp.P] = th[0], th[1]
        norm = np.concatenate([mu, sd]).astype(np.float32)
        sdd.sdd_cv_set_model(ctx, torch.from_numpy(block).cuda(), torch.from_numpy(norm).cuda(), S)
        sdd.sdd_cv_enable(ctx, sdd.SDD_CV_MODEL)
        mu, sd = norm[:5].astype(np.float64), norm[5:].astype(np.float64)
    else:
        sdd.sdd_cv_enable(ctx, sdd.SDD_CV_FIELDS)
    ii, jj = W.interface_nodes(n, n, sub, sub)
    state, gap = [xi0, eta0], 0.0
    for step in range(3):
        w = W.w_front(n, step * Dt)
        sdd.sdd_set_w(ctx, torch.from_numpy(w).cuda())
        sdd.sdd_step(ctx, dt=dt, Dt=Dt, seed=9, paths_per_node=paths, rtol=1e-13, max_iter=50000)
        sdd.sdd_sync(ctx)
        g = _np(sdd.sdd_last_interface_stats(ctx))
        if mode == "model":
            T = mlp.tabulate(th, mu, sd, w, K, S)
        else:
            T = _f(mlp.field_cell_gradient_table(*state, sdd.sdd_cv_fields_order(ctx)))
        new, o = oracle_mod.dd_step(w, state[0], state[1], sub_x=sub, sub_y=sub, dt=dt, Dt=Dt, n_paths=paths, seed=9,
                                    step_index=step, nodes_ij=(ii, jj), cv_table=T)
        se = {f: np.asarray(g["se_" + f]) + np.asarray(o["se_" + f]) for f in ("xi", "eta")}
        gfields = [a.cpu().numpy() for a in sdd.sdd_get_fields(ctx)]
        gap = PT.assert_trajectory_step(g, o, gfields, new, gap, slack=1e-4, se=se, tag=f"{mode} step {step}",
                                        clean=False)
        state = new


@pytest.mark.parametrize("mode", ["fields", "table"])
def test_zero_map_with_control_variate_changes_no_result(sdd, mode):
    # the control-variate kernels read the drift through the zero map too: every path record must be
    # the one the kernel without the map computes, bit for bit
    n = 257
    X, Y = W.grid(n)
    bump = np.exp(-((X - 0.5) ** 2 + (Y - 0.55) ** 2) / 0.01)
    xi0, eta0 = X + 0.01 * bump, Y - 0.008 * bump          # the identity mesh but near the middle
    ctx = _ctx(sdd, W.w_ring(n, 0.0), xi0, eta0)
    if mode == "fields":
        sdd.sdd_cv_enable(ctx, sdd.SDD_CV_FIELDS)
    else:
        from oracle import mlp
        _set_table(sdd, ctx, mlp.field_gradient_table(xi0, eta0))
        sdd.sdd_cv_enable(ctx, sdd.SDD_CV_TABLE)
    xs, ys = W.interface_node_coords(n, n, 2, 2)
    kw = dict(dt=1e-4, Dt=1e-2, seed=12, paths_per_task=128, block_threads=256)
    on = _np(sdd.sdd_interface_mc_record(ctx, xs, ys, 600, zero_map=1, **kw))
    off = _np(sdd.sdd_interface_mc_record(ctx, xs, ys, 600, zero_map=2, **kw))
    for k in on:
        np.testing.assert_array_equal(on[k], off[k], err_msg=k)


def test_field_cells_on_a_rectangular_grid_match_oracle(sdd, oracle_mod):
    # 65 x 41 nodes, fields with structure along both axes: the cell values of every order the
    # header admits at this size against the oracle's, and the paths' records with them
    from oracle import mlp
    nx, ny = 65, 41
    X, Y = W.grid(nx, ny)
    xi0 = X + 0.03 * np.sin(2 * np.pi * X) * np.sin(np.pi * Y) ** 2
    eta0 = Y + 0.02 * np.sin(np.pi * X) * np.sin(3 * np.pi * Y)
    w = (1.0 + 4.0 * np.exp(-((X - 0.6) ** 2 + (Y - 0.4) ** 2) / 0.02)).astype(np.float32)
    ctx = _ctx(sdd, w, xi0, eta0)
    sdd.sdd_cv_enable(ctx, sdd.SDD_CV_FIELDS)
    for order in (1, 3, 17, 255):
        sdd.sdd_cv_set_fields_order(ctx, order)
        C = mlp.field_cell_gradient_table(xi0, eta0, order)
        np.testing.assert_allclose(sdd.sdd_cv_get_cells(ctx).cpu().numpy(), C[0], rtol=0, atol=2e-6,
                                   err_msg=str(order))
    sdd.sdd_cv_set_fields_order(ctx, 17)
    xs, ys = W.interface_node_coords(nx, ny, 2, 2)
    npaths = np.full(xs.size, 400)
    kw = dict(dt=2e-4, Dt=1e-2, seed=3, exit_mode=0)
    g = _np(sdd.sdd_interface_mc_record(ctx, xs, ys, npaths, **kw))
    C = _f(mlp.field_cell_gradient_table(xi0, eta0, 17))
    o = oracle_mod.interface_mc(oracle_mod.Problem(w, xi0, eta0), xs, ys, npaths, record=True, cv_table=C, **kw)
    # the single-precision path can sit in a neighbouring cell of the oracle's for a sub-step (the
    # positions agree to ~1e-5, the cells here are 0.016 x 0.025 wide): each such sub-step moves a score
    # by at most the largest jump of the cell values between neighbouring cells times the increment
    # (below 5 standard deviations, sqrt(2 dt) 5); allow three per path
    jump = max(np.abs(np.diff(C[0], axis=0)).max(), np.abs(np.diff(C[0], axis=1)).max())
    tol = PT.PATH_TOL + 3 * jump * 5 * math.sqrt(2 * kw["dt"])
    assert tol < 0.05
    PT.assert_records(g, o, score_tol=tol)
    # the neighbouring-cell sub-steps move single scores either way: the node means still agree
    for f in ("xi", "eta"):
        d = np.abs(g["mean_" + f] - o["mean_" + f])
        assert np.all(d <= 3 * o["se_" + f] + 1e-12), (f, d.max())
        assert np.median(d) <= 1e-4, (f, np.median(d))
