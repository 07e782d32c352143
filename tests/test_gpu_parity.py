"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same Philox streams.

Tolerance (the estimator's own): per node within 3 standard errors of the
oracle's estimate; exit decisions identical for >= 99.9% of paths; paths with
identical exit decisions agree in score and end point to 1e-4; nodes whose
paths all agree agree in mean to 1e-4.
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


def _offsets(n_paths):
    return np.concatenate([[0], np.cumsum(n_paths)])


def _ctx(sdd, w, xi0=None, eta0=None, sub=2, faces=None):
    import torch
    ny, nx = w.shape
    wt = torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda()
    xt = torch.from_numpy(np.ascontiguousarray(xi0, np.float64)).cuda() if xi0 is not None else None
    et = torch.from_numpy(np.ascontiguousarray(eta0, np.float64)).cuda() if eta0 is not None else None
    ctx = sdd.sdd_init(nx, ny, sub, sub, w=wt, xi0=xt, eta0=et)
    if faces is not None:
        sdd.sdd_set_boundary(ctx, torch.from_numpy(np.ascontiguousarray(faces, np.float64)).cuda())
    return ctx


def test_rng_words_bit_exact_and_normals_close(sdd, oracle_mod):
    rng = np.random.default_rng(11)
    ctr = rng.integers(0, 2 ** 32, size=(200000, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4], [7, 0, 0, 1]]
    for seed in (0, 0x0123456789ABCDEF, 2 ** 64 - 1):
        wg, zg = sdd.sdd_rng_draw(seed, ctr)
        wo, zo = oracle_mod.draw(seed, ctr)
        np.testing.assert_array_equal(wg.cpu().numpy().view(np.uint32), wo)
        err = np.abs(zg.cpu().numpy().astype(np.float64) - zo)
        assert np.quantile(err, 0.9999) < 1e-5, np.quantile(err, 0.9999)
        assert err.max() < 2e-3, err.max()


@pytest.mark.parametrize("exit_mode", [0, 1])
def test_heat65_parity_and_closed_form(sdd, oracle_mod, exit_mode):
    xi0, eta0 = W.heat65_fields()
    faces = np.zeros(oracle_mod.faces_len(65, 65))
    ctx = _ctx(sdd, W.w_const(65), xi0, eta0, faces=faces)
    xs, ys = W.heat65_nodes()
    npaths = np.full(xs.size, 1000)
    g = _np(sdd.sdd_interface_mc_record(ctx, xs, ys, npaths, dt=1e-3, Dt=0.05, seed=0, exit_mode=exit_mode))
    P = oracle_mod.Problem(W.w_const(65), xi0, eta0, faces)
    o = oracle_mod.interface_mc(P, xs, ys, npaths, dt=1e-3, Dt=0.05, seed=0, exit_mode=exit_mode, record=True)
    same, rep = PT.assert_records(g, o)
    PT.assert_nodes(g, o, npaths, same, _offsets(npaths))
    if exit_mode == 0:
        PT.assert_flips_near_boundary(oracle_mod, P, xs, ys, npaths, g, o, same, dt=1e-3, Dt=0.05, seed=0)
    if exit_mode == 1:
        ex, ee = W.heat_exact(xs, ys, 0.05)
        inner = slice(1, 32)
        assert np.all(np.abs(g["mean_xi"] - ex)[inner] <= 3 * g["se_xi"][inner] + 3e-4)
        assert np.all(np.abs(g["mean_eta"] - ee)[inner] <= 3 * g["se_eta"][inner] + 3e-4)


def test_front257_full_size_sampled_nodes(sdd, oracle_mod):
    # the full 509-node, 1e4-path estimate at step 0 of the moving-front workload,
    # in the default launch shape; the oracle recomputes a sample of nodes
    n = 257
    w = W.w_front(n, 0.0)
    xi0, eta0 = W.identity_fields(n)
    ctx = _ctx(sdd, w, xi0, eta0)
    xs, ys = W.interface_node_coords(n, n, 2, 2)
    npaths = np.full(xs.size, 10000)
    g = _np(sdd.sdd_interface_mc_record(ctx, xs, ys, npaths, dt=1e-4, Dt=1e-2, seed=0, step_index=0))
    assert np.all((g["mean_xi"] > 0) & (g["mean_xi"] < 1) & (g["se_xi"] > 0))
    pick = np.array([0, 1, 2, 60, 127, 200, 253, 254, 255, 256, 300, 381, 450, 507, 508])
    P = oracle_mod.Problem(w, xi0, eta0)
    o = oracle_mod.interface_mc(P, xs[pick], ys[pick], 10000, dt=1e-4, Dt=1e-2, seed=0, step_index=0,
                                node_ids=pick.astype(np.uint32), record=True)
    off = _offsets(npaths)
    sel = np.concatenate([np.arange(off[k], off[k + 1]) for k in pick])
    gs = {k: g[k][sel] for k in ("steps", "code", "score_xi", "score_eta", "x_end", "y_end")}
    same, rep = PT.assert_records(gs, o)
    gn = {k: g[k][pick] for k in ("mean_xi", "mean_eta", "se_xi", "se_eta", "n_exit", "path_steps")}
    PT.assert_nodes(gn, o, np.full(pick.size, 10000), same, _offsets(np.full(pick.size, 10000)))
    PT.assert_flips_near_boundary(oracle_mod, P, xs[pick], ys[pick], 10000, gs, o, same, dt=1e-4, Dt=1e-2, seed=0,
                                  node_ids=pick)


@pytest.mark.parametrize("exit_mode", [0, 1])
@pytest.mark.parametrize("ppt", [0, 32, 96])
def test_ragged_nodes_and_launch_shapes(sdd, oracle_mod, exit_mode, ppt):
    n = 33
    w = W.w_smooth_random(n, 21)
    X, Y = W.grid(n)
    xi0 = X + 0.05 * np.sin(np.pi * X) * np.sin(2 * np.pi * Y)
    eta0 = Y.copy()
    ctx = _ctx(sdd, w, xi0, eta0, sub=3)
    xs = np.array([0.0, 1.0, 0.01, 0.5, 0.33, 0.999, 0.5, 0.72, 0.25])
    ys = np.array([0.3, 1.0, 0.5, 0.5, 0.004, 0.5, 0.98, 0.61, 0.5])
    npaths = np.array([37, 5, 1000, 64, 33, 1, 777, 31, 2])
    kw = dict(dt=1e-3, Dt=7e-3, seed=12345, step_index=9, exit_mode=exit_mode)
    g = _np(sdd.sdd_interface_mc_record(ctx, xs, ys, npaths, paths_per_task=ppt, **kw))
    P = oracle_mod.Problem(w, xi0, eta0)
    o = oracle_mod.interface_mc(P, xs, ys, npaths, record=True, **kw)
    same, rep = PT.assert_records(g, o)
    PT.assert_nodes(g, o, npaths, same, _offsets(npaths))
    if exit_mode == 0:
        PT.assert_flips_near_boundary(oracle_mod, P, xs, ys, npaths, g, o, same, dt=1e-3, Dt=7e-3, seed=12345,
                                      step_index=9)
    # boundary nodes: the Dirichlet value, zero SE, no steps, all paths counted as exits
    for k in (0, 1):
        assert g["se_xi"][k] == 0 and g["path_steps"][k] == 0 and g["n_exit"][k] == npaths[k]
        assert g["mean_xi"][k] == pytest.approx(o["mean_xi"][k], abs=1e-14)
        assert g["mean_eta"][k] == pytest.approx(o["mean_eta"][k], abs=1e-14)


def test_records_do_not_depend_on_launch_shape(sdd):
    n = 65
    ctx = _ctx(sdd, W.w_front(n, 0.3), *W.identity_fields(n))
    xs, ys = W.interface_node_coords(n, n, 2, 2)
    runs = []
    for ppt, block in ((0, 0), (32, 64), (160, 512), (2048, 128)):
        runs.append(_np(sdd.sdd_interface_mc_record(ctx, xs, ys, 700, dt=1e-4, Dt=1e-2, seed=3,
                                                    paths_per_task=ppt, block_threads=block)))
    for r in runs[1:]:
        for k in ("steps", "code", "score_xi", "score_eta", "x_end", "y_end"):
            np.testing.assert_array_equal(r[k], runs[0][k])
        # different lane groupings change only the single-precision lane sums
        np.testing.assert_allclose(r["mean_xi"], runs[0]["mean_xi"], rtol=0, atol=1e-8)
        np.testing.assert_array_equal(r["n_exit"], runs[0]["n_exit"])


def test_repeated_runs_are_bit_identical(sdd):
    n = 129
    ctx = _ctx(sdd, W.w_front(n, 0.1), *W.identity_fields(n))
    xs, ys = W.interface_node_coords(n, n, 2, 2)
    a = _np(sdd.sdd_interface_mc(ctx, xs, ys, 3000, dt=1e-4, Dt=1e-2, seed=5))
    b = _np(sdd.sdd_interface_mc(ctx, xs, ys, 3000, dt=1e-4, Dt=1e-2, seed=5))
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    c = _np(sdd.sdd_interface_mc(ctx, xs, ys, 3000, dt=1e-4, Dt=1e-2, seed=6))
    assert not np.array_equal(a["mean_xi"], c["mean_xi"])


def test_zero_map_changes_no_result(sdd):
    # where w is constant around a cell its drift records are zero and the path kernel of a
    # context reads the shared all-zero record instead (the zero map); the allocation-free entry
    # point runs the same kernel without the map: every output must be the same, bit for bit
    import torch
    n = 257
    for t, paths in ((0.0, 2000), (0.3, 701)):
        w = W.w_ring(n, t)
        # most of the square has w == 1 exactly (the map's case), the ring does not
        wd = w.astype(np.float64)
        flat = (wd[1:-1, 2:] == wd[1:-1, :-2]) & (wd[2:, 1:-1] == wd[:-2, 1:-1])
        assert 0.3 < flat.mean() < 0.95
        X, Y = W.identity_fields(n)
        ctx = _ctx(sdd, w, X, Y)
        xs, ys = W.interface_node_coords(n, n, 2, 2)
        kw = dict(dt=1e-4, Dt=1e-2, seed=9, step_index=2, paths_per_task=128, block_threads=256)
        a = _np(sdd.sdd_interface_mc(ctx, xs, ys, paths, **kw))
        b = _np(sdd.sdd_interface_mc_static(torch.from_numpy(w).cuda(), torch.from_numpy(X).cuda(),
                                            torch.from_numpy(Y).cuda(), xs, ys, paths, **kw))
        for k in a:
            np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_empty_and_single_path_nodes(sdd, oracle_mod):
    n = 17
    ctx = _ctx(sdd, W.w_const(n), *W.identity_fields(n))
    out = sdd.sdd_interface_mc(ctx, np.zeros(0), np.zeros(0), np.zeros(0, np.int64), dt=1e-3, Dt=1e-2)
    assert out["mean_xi"].numel() == 0
    g = _np(sdd.sdd_interface_mc(ctx, [0.5, 0.2], [0.5, 0.9], [1, 1], dt=1e-3, Dt=1e-3))  # K = 1
    P = oracle_mod.Problem(W.w_const(n), *W.identity_fields(n))
    o = oracle_mod.interface_mc(P, [0.5, 0.2], [0.5, 0.9], [1, 1], dt=1e-3, Dt=1e-3)
    np.testing.assert_allclose(g["mean_xi"], o["mean_xi"], atol=1e-6)
    assert np.all(g["se_xi"] == 0)


def test_host_side_rejections(sdd):
    n = 17
    ctx = _ctx(sdd, W.w_const(n), *W.identity_fields(n))
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_interface_mc(ctx, [0.5], [0.5], [10], dt=3e-3, Dt=1e-2)    # Dt / dt not an integer
    assert e.value.status == sdd.SDD_EINVAL
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_interface_mc(ctx, [1.5], [0.5], [10], dt=1e-3, Dt=1e-2)    # node outside
    assert e.value.status == sdd.SDD_EINVAL
    with pytest.raises(sdd.SddError):
        sdd.sdd_interface_mc(ctx, [0.5], [0.5], [0], dt=1e-3, Dt=1e-2)     # no paths
    with pytest.raises(sdd.SddError):
        sdd.sdd_interface_mc(ctx, [0.5], [0.5], [10], dt=1e-3, Dt=1e-2, exit_mode=3)    # no such exit test
    with pytest.raises(sdd.SddError):
        sdd.sdd_interface_mc(ctx, [0.5], [0.5], [10], dt=1e-3, Dt=1e-2, paths_per_task=48)
    sdd.sdd_sync(ctx)


def test_nonpositive_w_is_reported_by_sync(sdd):
    import torch
    n = 17
    ctx = _ctx(sdd, W.w_const(n), *W.identity_fields(n))
    w = torch.ones((n, n), dtype=torch.float32, device="cuda")
    w[5, 7] = 0.0
    sdd.sdd_set_w(ctx, w)
    sdd.sdd_interface_mc(ctx, [0.5], [0.5], [100], dt=1e-3, Dt=1e-2)
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_sync(ctx)
    assert e.value.status == sdd.SDD_EDEVICE
    sdd.sdd_set_w(ctx, torch.ones((n, n), dtype=torch.float32, device="cuda"))
    sdd.sdd_interface_mc(ctx, [0.5], [0.5], [100], dt=1e-3, Dt=1e-2)
    sdd.sdd_sync(ctx)


def test_faces_match_oracle(sdd, oracle_mod):
    n = 129
    w = W.w_front(n, 0.2) * W.w_bump(n, 0.3, 0.6, 0.1, 3.0)
    ctx = _ctx(sdd, w, *W.identity_fields(n))
    g = sdd.sdd_get_faces(ctx).cpu().numpy()
    o = oracle_mod.winslow_faces(w.astype(np.float64))
    np.testing.assert_allclose(g, o, rtol=0, atol=1e-14)


def test_interface_node_order(sdd):
    n = 65
    ctx = _ctx(sdd, W.w_const(n), *W.identity_fields(n), sub=4)
    x, y = sdd.sdd_interface_nodes(ctx)
    wx, wy = W.interface_node_coords(n, n, 4, 4)
    np.testing.assert_array_equal(x, wx)
    np.testing.assert_array_equal(y, wy)


def test_subdomain_solve_matches_lu(sdd, oracle_mod):
    from oracle import solver
    import torch
    n = 41
    w = W.w_smooth_random(n, 8) * W.w_bump(n, 0.6, 0.4, 0.15, 4.0)
    X, Y = W.grid(n)
    prev = [X + 0.03 * np.sin(2 * np.pi * X) * np.sin(np.pi * Y), Y + 0.02 * np.sin(np.pi * X)]
    ctx = _ctx(sdd, w, prev[0], prev[1])
    ii, jj = W.interface_nodes(n, n, 2, 2)
    rng = np.random.default_rng(2)
    vx = X[jj, ii] + rng.normal(0, 1e-3, ii.size)
    ve = Y[jj, ii] + rng.normal(0, 1e-3, ii.size)
    Dt = 5e-3
    gx, ge, iters = sdd.sdd_subdomain_solve(ctx, Dt, torch.from_numpy(vx).cuda(), torch.from_numpy(ve).cuda(),
                                            rtol=1e-13, max_iter=20000)
    assert 0 < iters < 20000
    faces = oracle_mod.winslow_faces(w.astype(np.float64))
    bx = oracle_mod.boundary_grid(faces, n, n, 0, prev[0])
    be = oracle_mod.boundary_grid(faces, n, n, 1, prev[1])
    bx[jj, ii] = vx
    be[jj, ii] = ve
    ox, oe = solver.subdomain_solve(w.astype(np.float64), prev, [bx, be], 2, 2, Dt)
    np.testing.assert_allclose(gx.cpu().numpy(), ox, rtol=0, atol=1e-10)
    np.testing.assert_allclose(ge.cpu().numpy(), oe, rtol=0, atol=1e-10)


def test_solver_nonconvergence_is_a_status(sdd):
    import torch
    n = 33
    ctx = _ctx(sdd, W.w_smooth_random(n, 1), *W.identity_fields(n))
    sdd.sdd_set_solver(ctx, sdd.SDD_SOLVER_JACOBI)
    x, y = sdd.sdd_interface_nodes(ctx)
    v = torch.from_numpy(x + 0.01).cuda()
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_subdomain_solve(ctx, 1e-2, v, v, rtol=1e-14, max_iter=3)
    assert e.value.status == sdd.SDD_ENOCONV


def test_mesh_steps_match_oracle(sdd, oracle_mod):
    # three mesh steps through sdd_step against three steps of the oracle (its Monte Carlo
    # estimate, then its LU subdomain solves, Sec. 4) from the same seeded start, each side on
    # its own fields: the allowance for the previous fields' gap is the gap itself, and the
    # solve's maximum principle bounds the new gap by the interface values' (R14)
    import torch
    n, sub = 65, 2
    dt, Dt, paths = 1e-4, 1e-2, 4000
    xi, eta = W.identity_fields(n)
    ctx = _ctx(sdd, W.w_front(n, 0.0), xi, eta, sub=sub)
    ii, jj = W.interface_nodes(n, n, sub, sub)
    state, gap = [xi, eta], 0.0
    for step in range(3):
        w = W.w_front(n, step * Dt)
        sdd.sdd_set_w(ctx, torch.from_numpy(w).cuda())
        sdd.sdd_step(ctx, dt=dt, Dt=Dt, seed=77, paths_per_node=paths, rtol=1e-13, max_iter=50000)
        sdd.sdd_sync(ctx)
        g = _np(sdd.sdd_last_interface_stats(ctx))
        gfields = [a.cpu().numpy() for a in sdd.sdd_get_fields(ctx)]
        new, o = oracle_mod.dd_step(w, state[0], state[1], sub_x=sub, sub_y=sub, dt=dt, Dt=Dt, n_paths=paths,
                                    seed=77, step_index=step, nodes_ij=(ii, jj))
        np.testing.assert_array_equal(g["path_steps"] > 0, o["path_steps"] > 0)
        gap = PT.assert_trajectory_step(g, o, gfields, new, gap, tag=f"step {step}")
        state = new
    assert sdd.sdd_get_step_index(ctx) == 3


def test_autotune_chooses_a_candidate_and_keeps_results(sdd):
    n = 129
    ctx = _ctx(sdd, W.w_front(n, 0.15), *W.identity_fields(n))
    xs, ys = W.interface_node_coords(n, n, 2, 2)
    kw = dict(dt=1e-4, Dt=1e-2)
    before = _np(sdd.sdd_interface_mc_record(ctx, xs, ys, 2000, seed=21, **kw))
    shape = sdd.sdd_autotune(ctx, xs, ys, 2000, **kw)
    assert shape["block_threads"] in (128, 256, 512)
    assert shape["paths_per_task"] in (32, 64, 128, 256, 512, 1024) and shape["ms"] > 0
    after = _np(sdd.sdd_interface_mc_record(ctx, xs, ys, 2000, seed=21, **kw))
    for k in ("steps", "code", "score_xi", "x_end"):
        np.testing.assert_array_equal(after[k], before[k])
    np.testing.assert_allclose(after["mean_xi"], before["mean_xi"], rtol=0, atol=1e-8)
    # a tuned mesh step runs and advances the counter
    sdd.sdd_step(ctx, dt=1e-4, Dt=1e-2, seed=1, paths_per_node=500, tune=1)
    sdd.sdd_sync(ctx)
    assert sdd.sdd_get_step_index(ctx) == 1
