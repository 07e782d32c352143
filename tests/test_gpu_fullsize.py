"""Full-size parity in the launch configuration the bench times: mesh steps through
sdd_step (tuned launch shape, CUDA graph, pipelined solve with deferred survivor
scoring where it applies), compared with the FP64 oracle at sampled interface
nodes on the same Philox streams.

Tolerance (the estimator's own): per node within 3 standard errors of the
oracle's estimate; the sampled nodes' median deviation far below one standard
error (identical streams: only rare exit flips and single-precision rounding
separate them); exit and path-step counts within 0.1% of the oracle's.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sdd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1402_0266_gb300 import build
    build.build()
    import paper_1402_0266_gb300 as m
    return m


def _ctx(sdd, n, sub, w0):
    import torch
    xi, eta = W.identity_fields(n)
    return sdd.sdd_init(n, n, sub, sub, w=torch.from_numpy(np.ascontiguousarray(w0, np.float32)).cuda(),
                        xi0=torch.from_numpy(xi).cuda(), eta0=torch.from_numpy(eta).cuda())


def _stats(sdd, ctx):
    return {k: v.cpu().numpy() for k, v in sdd.sdd_last_interface_stats(ctx).items()}


def _path_by_path(sdd, oracle_mod, P, fields, w, xs, ys, pick, paths, dt, Dt, step, g, field_gap=0.0):
    """The sampled nodes once more, each on its own context with the GPU's w and fields and its own
    node word, through the per-path record entry point: its records against the oracle's path by
    path (P: the oracle's problem, on the oracle's own fields; they differ from the GPU's by at most
    field_gap, by which a surviving path's score may then differ), and its node results against the
    step's (the step scored its paths in another kernel and summed them in another order)."""
    import torch
    from tests import _parity as PT
    n = w.shape[0]
    c = sdd.sdd_init(n, n, 1, 1, w=torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda(),
                     xi0=torch.from_numpy(fields[0]).cuda(), eta0=torch.from_numpy(fields[1]).cuda())
    for k, node in enumerate(pick):
        x, y = xs[node:node + 1], ys[node:node + 1]
        r = {key: v.cpu().numpy() for key, v in sdd.sdd_interface_mc_record(
            c, x, y, [paths], dt=dt, Dt=Dt, seed=0, step_index=step, node_word0=int(node)).items()}
        o = oracle_mod.interface_mc(P, x, y, paths, dt=dt, Dt=Dt, seed=0, step_index=step,
                                    node_ids=np.array([node], np.uint32), record=True)
        same, rep = PT.assert_records(r, o, score_tol=PT.PATH_TOL + field_gap)
        PT.assert_flips_near_boundary(oracle_mod, P, x, y, [paths], r, o, same, dt=dt, Dt=Dt, seed=0,
                                      step_index=step, node_ids=np.array([node], np.uint32))
        for f in ("xi", "eta"):
            assert abs(r["mean_" + f][0] - g["mean_" + f][node]) <= 1e-6, (node, f)
            assert abs(r["se_" + f][0] - g["se_" + f][node]) <= 1e-6 * max(1.0, g["se_" + f][node]), (node, f)
        for key in ("n_exit", "path_steps"):
            assert r[key][0] == g[key][node], (node, key)


def _compare(g, o, pick, field_gap=0.0):
    # field_gap: the largest difference between the GPU's and the oracle's previous fields, which a
    # surviving path's score inherits
    for f in ("xi", "eta"):
        d = np.abs(g["mean_" + f][pick] - o["mean_" + f])
        assert np.all(d <= 3 * o["se_" + f] + field_gap), (f, d.max(), (d / o["se_" + f]).max())
        assert np.median(np.maximum(d - field_gap, 0) / o["se_" + f]) < 0.1, (f, np.median(d / o["se_" + f]))
        np.testing.assert_allclose(g["se_" + f][pick], o["se_" + f], rtol=2e-2)
    for k in ("n_exit", "path_steps"):
        np.testing.assert_allclose(g[k][pick], o[k], rtol=1e-3)


def test_front257_pipelined_steps_full_size_sampled_nodes(sdd, oracle_mod):
    import torch
    n, Dt, dt, paths = 257, 1e-2, 1e-4, 10000
    kw = dict(dt=dt, Dt=Dt, seed=0, paths_per_node=paths, rtol=1e-12, max_iter=20000, tune=1)
    w = [W.w_front(n, k * Dt) for k in range(2)]
    # A: two steps back to back (the second runs the first's solve beside its paths, then scores its
    # survivors and exits from their records once the new fields are final); the fields between
    # them read out (which enqueues the pending iterations early and changes no result)
    a = _ctx(sdd, n, 2, w[0])
    sdd.sdd_set_w(a, torch.from_numpy(w[0]).cuda())
    sdd.sdd_step(a, **kw)
    fa1 = [t.cpu().numpy() for t in sdd.sdd_get_fields(a)]
    sdd.sdd_set_w(a, torch.from_numpy(w[1]).cuda())
    sdd.sdd_step(a, **kw)
    assert sdd.sdd_pipeline_in_use(a)
    a2 = _stats(sdd, a)
    # B: one step, then its fields (the first step's solve flushed)
    b = _ctx(sdd, n, 2, w[0])
    sdd.sdd_set_w(b, torch.from_numpy(w[0]).cuda())
    sdd.sdd_step(b, **kw)
    b1 = _stats(sdd, b)
    f1 = [t.cpu().numpy() for t in sdd.sdd_get_fields(b)]
    sdd.sdd_sync(a)
    sdd.sdd_sync(b)
    xs, ys = W.interface_node_coords(n, n, 2, 2)
    pick = np.array([0, 3, 64, 127, 190, 252, 254, 256, 320, 381, 444, 505, 508])
    xi0, eta0 = W.identity_fields(n)
    # the oracle's own first mesh step (estimate at every node, LU solves): its fields start its
    # second step, as the GPU's start the GPU's
    ii, jj = W.interface_nodes(n, n, 2, 2)
    of1, o1 = oracle_mod.dd_step(w[0], xi0, eta0, sub_x=2, sub_y=2, dt=dt, Dt=Dt, n_paths=paths, seed=0, step_index=0,
                                 nodes_ij=(ii, jj))
    _compare(b1, {k: v[pick] for k, v in o1.items() if np.ndim(v) == 1 and len(v) == xs.size}, pick)
    gap = max(float(np.abs(f[k] - of1[k]).max()) for f in (fa1, f1) for k in (0, 1))
    iface = max(float(np.abs(b1["mean_xi"] - o1["mean_xi"]).max()), float(np.abs(b1["mean_eta"] - o1["mean_eta"]).max()))
    assert gap <= iface + 1e-9, (gap, iface)                   # the solve's maximum principle (R14)
    P2 = oracle_mod.Problem(w[1], of1[0], of1[1])
    o2 = oracle_mod.interface_mc(P2, xs[pick], ys[pick], paths, dt=dt, Dt=Dt, seed=0, step_index=1,
                                 node_ids=pick.astype(np.uint32))
    _compare(a2, o2, pick, gap)
    # the deferred scoring of the pipelined step, path by path (seven of the sampled nodes)
    sub_pick = pick[::2]
    _path_by_path(sdd, oracle_mod, P2, fa1, w[1], xs, ys, sub_pick, paths, dt, Dt, 1, a2, gap)


def test_ring2049_step_full_size_sampled_nodes(sdd, oracle_mod):
    import torch
    n, sub, Dt, dt, paths = 2049, 8, 1e-3, 1e-5, 20000
    w0 = W.w_ring(n, 0.0)
    c = _ctx(sdd, n, sub, w0)
    sdd.sdd_set_w(c, torch.from_numpy(w0).cuda())
    sdd.sdd_step(c, dt=dt, Dt=Dt, seed=0, paths_per_node=paths, rtol=1e-12, max_iter=20000, tune=1)
    g = _stats(sdd, c)
    sdd.sdd_sync(c)
    xs, ys = W.interface_node_coords(n, n, sub, sub)
    # nodes on the ring (steep w), between rings, at crossings and next to the boundary
    r = np.hypot(xs - 0.5, ys - 0.5)
    on_ring = np.flatnonzero(np.abs(r - 0.25) < 2e-3)[:4]
    pick = np.unique(np.concatenate([on_ring, [0, 1, 1023, 2046, 14000, 28607, 28608]]))
    xi0, eta0 = W.identity_fields(n)
    P = oracle_mod.Problem(w0, xi0, eta0)
    o = oracle_mod.interface_mc(P, xs[pick], ys[pick], paths, dt=dt, Dt=Dt, seed=0, step_index=0,
                                node_ids=pick.astype(np.uint32))
    _compare(g, o, pick)
    # the step's deferred scoring, path by path, at four of the sampled nodes
    _path_by_path(sdd, oracle_mod, P, (xi0, eta0), w0, xs, ys, pick[[0, 2, 5, -1]], paths, dt, Dt, 0, g)


def test_ring2049_field_gradient_control_variate_full_size_sampled_nodes(sdd, oracle_mod):
    # the control-variate path kernel at full size (2049^2 cell tables, the zero map, the smoothed
    # cell values of the fields): records of sampled nodes path by path against the oracle's with
    # the same model computed from the same seeded fields
    import torch
    from oracle import mlp
    from tests import _parity as PT
    n, sub, Dt, dt, paths = 2049, 8, 1e-3, 1e-5, 4000
    X, Y = W.grid(n)
    r = np.hypot(X - 0.5, Y - 0.5)
    bump = np.exp(-((r - 0.25) / 0.05) ** 2)
    xi0 = X + 0.01 * (X - 0.5) * bump                   # a mesh pulled towards the ring
    eta0 = Y + 0.01 * (Y - 0.5) * bump
    w0 = W.w_ring(n, 0.0)
    c = sdd.sdd_init(n, n, sub, sub, w=torch.from_numpy(w0).cuda(), xi0=torch.from_numpy(xi0).cuda(),
                     eta0=torch.from_numpy(eta0).cuda())
    sdd.sdd_cv_enable(c, sdd.SDD_CV_FIELDS)
    order = sdd.sdd_cv_fields_order(c)
    assert order == 33
    C = mlp.field_cell_gradient_table(xi0, eta0, order)
    np.testing.assert_allclose(sdd.sdd_cv_get_cells(c).cpu().numpy(), C[0], rtol=0, atol=2e-6)
    xs, ys = W.interface_node_coords(n, n, sub, sub)
    rr = np.hypot(xs - 0.5, ys - 0.5)
    pick = np.unique(np.concatenate([np.flatnonzero(np.abs(rr - 0.25) < 2e-3)[:2], [5, 14000, 28600]]))
    P = oracle_mod.Problem(w0, xi0, eta0)
    Cf = np.asarray(C, np.float32).astype(np.float64)
    jump = max(np.abs(np.diff(Cf[0], axis=0)).max(), np.abs(np.diff(Cf[0], axis=1)).max())
    tol = PT.PATH_TOL + 3 * jump * 5 * np.sqrt(2 * dt)          # neighbouring-cell sub-steps, as on 65 x 41
    for node in pick:
        x, y = xs[node:node + 1], ys[node:node + 1]
        g = {k: v.cpu().numpy() for k, v in sdd.sdd_interface_mc_record(
            c, x, y, [paths], dt=dt, Dt=Dt, seed=3, node_word0=int(node)).items()}
        o = oracle_mod.interface_mc(P, x, y, paths, dt=dt, Dt=Dt, seed=3, node_ids=np.array([node], np.uint32),
                                    record=True, cv_table=Cf)
        PT.assert_records(g, o, score_tol=tol)
        for f in ("xi", "eta"):
            assert abs(g["mean_" + f][0] - o["mean_" + f][0]) <= 3 * o["se_" + f][0] + 1e-12, (node, f)
