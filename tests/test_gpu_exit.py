"""Exit tests and exponential time-stepping on the GPU against the oracle (Sec. 4 and its
"more sophisticated boundary tests" / "exponential time-stepping" alternatives)."""
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


@pytest.mark.parametrize("dt,Dt", [(1e-3, 2e-2), (2.5e-4, 1e-2)])
def test_exponential_time_stepping_records_match_oracle(sdd, oracle_mod, dt, Dt):
    n = 65
    w = W.w_front(n, 0.3)
    X, Y = W.grid(n)
    xi0 = X + 0.02 * np.sin(np.pi * X) * np.sin(np.pi * Y)
    eta0 = Y.copy()
    ctx = _ctx(sdd, w, xi0, eta0)
    xs, ys = W.interface_node_coords(n, n, 2, 2)
    pick = np.arange(0, xs.size, 6)
    xs = np.concatenate([xs[pick], [0.0, 0.02, 0.5]])
    ys = np.concatenate([ys[pick], [0.3, 0.5, 0.995]])
    npaths = np.full(xs.size, 600)
    npaths[::4] = 29
    kw = dict(dt=dt, Dt=Dt, seed=21, step_index=3, exit_mode=2)
    g = _np(sdd.sdd_interface_mc_record(ctx, xs, ys, npaths, **kw))
    o = oracle_mod.interface_mc(oracle_mod.Problem(w, xi0, eta0), xs, ys, npaths, record=True, **kw)
    # every sub-step adds a single-precision logarithm (its length) to the path, so end points agree to
    # the usual 1e-4 and scores to 1e-4 times the face data's slope (up to ~7 on this front): 3e-4
    same, rep = PT.assert_records(g, o, score_tol=3e-4)
    assert rep["max_x_end"] <= 1e-4 and rep["max_y_end"] <= 1e-4
    nodes_ok = np.array([same[a:b].all() for a, b in zip(np.concatenate([[0], np.cumsum(npaths)])[:-1],
                                                           np.cumsum(npaths))])
    for f in ("xi", "eta"):
        d = np.abs(g["mean_" + f] - o["mean_" + f])
        assert np.all(d <= 3 * o["se_" + f] + 3e-4 * nodes_ok), (f, d.max())
    # random sub-step counts: surviving paths take K + 1 on average
    K = int(round(Dt / dt))
    surv = g["code"] == -1
    assert abs(g["steps"][surv].mean() - (K + 1)) < 0.1 * (K + 1)


def test_exponential_time_stepping_heat_closed_form(sdd, oracle_mod):
    xi0, eta0 = W.heat65_fields()
    faces = np.zeros(oracle_mod.faces_len(65, 65))
    ctx = _ctx(sdd, W.w_const(65), xi0, eta0, faces=faces)
    xs, ys = W.heat65_nodes()
    xs, ys = xs[1:32], ys[1:32]
    g = _np(sdd.sdd_interface_mc(ctx, xs, ys, np.full(xs.size, 200000), dt=1e-2, Dt=0.05, seed=5, exit_mode=2))
    ex, ee = W.heat_exact(xs, ys, 0.05)
    assert np.all(np.abs(g["mean_xi"] - ex) <= 4 * g["se_xi"] + 3e-4), np.abs(g["mean_xi"] - ex) / g["se_xi"]
    assert np.all(np.abs(g["mean_eta"] - ee) <= 4 * g["se_eta"] + 3e-4)


def test_exponential_time_stepping_mesh_step_and_rejections(sdd, oracle_mod):
    import torch
    n, sub, dt, Dt, paths = 33, 2, 2.5e-4, 1e-2, 1500
    w = W.w_front(n, 0.0)
    xi, eta = W.identity_fields(n)
    ctx = _ctx(sdd, w, xi, eta, sub)
    sdd.sdd_step(ctx, dt=dt, Dt=Dt, seed=9, paths_per_node=paths, exit_mode=2, rtol=1e-13, max_iter=50000)
    sdd.sdd_sync(ctx)
    g = _np(sdd.sdd_last_interface_stats(ctx))
    ii, jj = W.interface_nodes(n, n, sub, sub)
    new, o = oracle_mod.dd_step(w, xi, eta, sub_x=sub, sub_y=sub, dt=dt, Dt=Dt, n_paths=paths, seed=9,
                                step_index=0, nodes_ij=(ii, jj), exit_mode=2)
    for f in ("xi", "eta"):
        d = np.abs(g["mean_" + f] - o["mean_" + f])
        assert np.all(d <= 3 * o["se_" + f] + 1e-4), (f, d.max())
    gx, ge = (a.cpu().numpy() for a in sdd.sdd_get_fields(ctx))
    iface_gap = max(np.abs(g["mean_xi"] - o["mean_xi"]).max(), np.abs(g["mean_eta"] - o["mean_eta"]).max())
    assert max(np.abs(gx - new[0]).max(), np.abs(ge - new[1]).max()) <= iface_gap + 1e-9
    # the control variate needs fixed sub-steps; unknown modes are rejected
    sdd.sdd_cv_enable(ctx, sdd.SDD_CV_FIELDS)
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_interface_mc(ctx, [0.5], [0.5], [10], dt=dt, Dt=Dt, exit_mode=2)
    assert e.value.status == sdd.SDD_EINVAL
    sdd.sdd_cv_enable(ctx, sdd.SDD_CV_OFF)
    with pytest.raises(sdd.SddError):
        sdd.sdd_interface_mc(ctx, [0.5], [0.5], [10], dt=dt, Dt=Dt, exit_mode=3)
