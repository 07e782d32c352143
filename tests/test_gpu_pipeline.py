"""Pipelined mesh steps: the subdomain solve of step n runs beside the paths of
step n + 1, whose survivors are scored once the new fields are final.

The pipelined sequence computes what the unpipelined one does; only the order
of the single-precision sums over a task's paths differs (the survivors' scores
are summed apart from the exits'), so interface means and fields agree to a few
units of single-precision rounding of those sums, and the integer counts
exactly. Flushing the pending iterations between steps changes nothing at all.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 2e-6   # single-precision rounding of the per-lane sums, over at most 1e4 paths per node


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


def _run(sdd, ctx, n, steps, kw, sync_every=False):
    """steps mesh steps of the moving front; returns the last step's statistics and the fields."""
    import torch
    for k in range(steps):
        sdd.sdd_set_w(ctx, torch.from_numpy(W.w_front(n, k * kw["Dt"])).cuda())
        sdd.sdd_step(ctx, **kw)
        if sync_every:
            sdd.sdd_sync(ctx)
    st = {k: v.cpu().numpy() for k, v in sdd.sdd_last_interface_stats(ctx).items()}
    gx, ge = (a.cpu().numpy() for a in sdd.sdd_get_fields(ctx))
    sdd.sdd_sync(ctx)
    return st, gx, ge


def _set_cv_table(sdd, ctx, n, slices, seed):
    import torch
    rng = np.random.default_rng(seed)
    g = rng.normal(0.0, 0.3, size=(slices, n, n, 4))
    sdd.sdd_cv_set_table(ctx, torch.from_numpy(g).cuda())
    sdd.sdd_cv_enable(ctx, sdd.SDD_CV_TABLE)


@pytest.mark.parametrize("n,sub,solver,exit_mode,cv,keypoints", [
    (65, 2, "auto", 0, False, False),     # register-resident Jacobi-PCG
    (65, 2, "auto", 1, False, False),     # bridge test
    (65, 2, "auto", 2, False, False),     # exponential time-stepping
    (65, 2, "auto", 0, True, False),      # control variate from a table: float4 survivor records
    (129, 2, "mg", 0, False, True),       # cluster multigrid, key points only
    (257, 2, "auto", 0, False, False),    # the cluster multigrid of the 257^2 front
])
def test_pipelined_steps_match_unpipelined(sdd, n, sub, solver, exit_mode, cv, keypoints):
    kw = dict(dt=1e-4, Dt=1e-2, seed=9, paths_per_node=3000, exit_mode=exit_mode, rtol=1e-12, max_iter=20000)
    out = []
    for pipe in (True, False):
        ctx = _ctx(sdd, n, sub, W.w_front(n, 0.0))
        if solver == "mg":
            sdd.sdd_set_solver(ctx, sdd.SDD_SOLVER_MG)
        if cv:
            _set_cv_table(sdd, ctx, n, 2, 3)
        if keypoints:
            sdd.sdd_set_keypoints(ctx, True, 8)
        sdd.sdd_set_pipeline(ctx, pipe)
        out.append(_run(sdd, ctx, n, 4, kw))
        assert sdd.sdd_pipeline_in_use(ctx) == pipe
        assert sdd.sdd_get_step_index(ctx) == 4
    (a, ax, ae), (b, bx, be) = out
    for k in ("n_exit", "path_steps"):
        np.testing.assert_array_equal(a[k], b[k])
    for k in ("mean_xi", "mean_eta"):
        np.testing.assert_allclose(a[k], b[k], rtol=0, atol=TOL)
    for k in ("se_xi", "se_eta"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-4, atol=1e-9)
    np.testing.assert_allclose(ax, bx, rtol=0, atol=TOL)
    np.testing.assert_allclose(ae, be, rtol=0, atol=TOL)
    # the estimate moved the fields: the comparison is not between two unchanged grids
    xi0, _ = W.identity_fields(n)
    assert np.abs(ax - xi0).max() > 1e-3


def test_flush_between_steps_changes_nothing(sdd):
    n = 129
    kw = dict(dt=1e-4, Dt=1e-2, seed=4, paths_per_node=2000, rtol=1e-12, max_iter=20000)
    a = _run(sdd, _ctx(sdd, n, 2, W.w_front(n, 0.0)), n, 4, kw, sync_every=False)
    b = _run(sdd, _ctx(sdd, n, 2, W.w_front(n, 0.0)), n, 4, kw, sync_every=True)
    for k in a[0]:
        np.testing.assert_array_equal(a[0][k], b[0][k])
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[2])


def test_field_gradient_control_variate_is_not_pipelined(sdd):
    n = 65
    ctx = _ctx(sdd, n, 2, W.w_front(n, 0.0))
    sdd.sdd_cv_enable(ctx, sdd.SDD_CV_FIELDS)
    _run(sdd, ctx, n, 2, dict(dt=1e-4, Dt=1e-2, seed=1, paths_per_node=500))
    assert not sdd.sdd_pipeline_in_use(ctx)


def test_reads_between_steps_see_final_fields(sdd):
    """sdd_get_fields and a direct estimate both come after the pending solve."""
    n = 65
    kw = dict(dt=1e-4, Dt=1e-2, seed=2, paths_per_node=1000)
    ref = _ctx(sdd, n, 2, W.w_front(n, 0.0))
    sdd.sdd_set_pipeline(ref, False)
    ctx = _ctx(sdd, n, 2, W.w_front(n, 0.0))
    for c in (ref, ctx):
        sdd.sdd_step(c, **kw)
        sdd.sdd_step(c, **kw)
    assert sdd.sdd_pipeline_in_use(ctx)
    xs, ys = sdd.sdd_interface_nodes(ctx)
    g = {k: v.cpu().numpy() for k, v in sdd.sdd_interface_mc(ctx, xs, ys, 800, dt=1e-4, Dt=1e-2, seed=5).items()}
    r = {k: v.cpu().numpy() for k, v in sdd.sdd_interface_mc(ref, xs, ys, 800, dt=1e-4, Dt=1e-2, seed=5).items()}
    np.testing.assert_array_equal(g["path_steps"], r["path_steps"])
    np.testing.assert_allclose(g["mean_xi"], r["mean_xi"], rtol=0, atol=TOL)
    fx, _ = (a.cpu().numpy() for a in sdd.sdd_get_fields(ctx))
    rx, _ = (a.cpu().numpy() for a in sdd.sdd_get_fields(ref))
    np.testing.assert_allclose(fx, rx, rtol=0, atol=TOL)
    # the step info of a pipelined step counts the deferred iterations as solve time
    sdd.sdd_step(ctx, **kw)
    sdd.sdd_step(ctx, **kw)
    info = sdd.sdd_last_step_info(ctx)
    assert info["solve_ms"] > 0 and info["paths_ms"] > 0 and info["kernel_nodes"] > 0
    sdd.sdd_sync(ctx)


def test_batch_after_pipelined_steps_sees_final_fields(sdd):
    """A context stepped on its own (pipelined) and then put into a batch: the batch
    runs the pending iterations first, so its estimate starts from the same fields as
    a context that was synchronised before."""
    import torch
    n = 65
    kw = dict(dt=1e-4, Dt=1e-2, seed=3, paths_per_node=800)
    a = _ctx(sdd, n, 2, W.w_front(n, 0.0))
    b = _ctx(sdd, n, 2, W.w_front(n, 0.0))
    for c in (a, b):
        for k in range(2):
            sdd.sdd_set_w(c, torch.from_numpy(W.w_front(n, k * 1e-2)).cuda())
            sdd.sdd_step(c, **kw)
    assert sdd.sdd_pipeline_in_use(a)
    sdd.sdd_sync(b)                                   # b's pending solve runs here
    batch = sdd.sdd_batch_create([a])                 # a's runs here
    sdd.sdd_batch_sync(batch)
    fa = [t.cpu().numpy() for t in sdd.sdd_get_fields(a)]
    fb = [t.cpu().numpy() for t in sdd.sdd_get_fields(b)]
    np.testing.assert_array_equal(fa[0], fb[0])
    np.testing.assert_array_equal(fa[1], fb[1])
    xs, ys = sdd.sdd_interface_nodes(a)
    est = sdd.sdd_batch_interface_mc(batch, [(xs, ys, np.full(xs.size, 500))], dt=1e-4, Dt=1e-2, seed=8)
    ref = sdd.sdd_interface_mc(b, xs, ys, np.full(xs.size, 500), dt=1e-4, Dt=1e-2, seed=8)
    sdd.sdd_batch_sync(batch)
    np.testing.assert_allclose(est[0]["mean_xi"].cpu().numpy(), ref["mean_xi"].cpu().numpy(), rtol=0, atol=1e-6)
    sdd.sdd_batch_destroy(batch)


def test_changed_parameters_flush_the_pending_solve(sdd):
    """New step parameters rebuild the step graphs; the last step's deferred
    iterations run first, so the sequence matches the unpipelined one."""
    import torch
    n = 65
    seq = [dict(dt=1e-4, Dt=1e-2, seed=1, paths_per_node=600),
           dict(dt=1e-4, Dt=1e-2, seed=1, paths_per_node=600),
           dict(dt=2e-4, Dt=1e-2, seed=2, paths_per_node=900, exit_mode=1),
           dict(dt=2e-4, Dt=1e-2, seed=2, paths_per_node=900, exit_mode=1)]
    out = []
    for pipe in (True, False):
        c = _ctx(sdd, n, 2, W.w_front(n, 0.0))
        sdd.sdd_set_pipeline(c, pipe)
        for k, kw in enumerate(seq):
            sdd.sdd_set_w(c, torch.from_numpy(W.w_front(n, k * 1e-2)).cuda())
            sdd.sdd_step(c, **kw)
        out.append([t.cpu().numpy() for t in sdd.sdd_get_fields(c)])
        sdd.sdd_sync(c)
    np.testing.assert_allclose(out[0][0], out[1][0], rtol=0, atol=TOL)
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=0, atol=TOL)
