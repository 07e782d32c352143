"""The multigrid-preconditioned subdomain solver against the oracle's sparse LU (Sec. 4's
"LU-factorization" of the implicit step), on decompositions whose subdomains coarsen."""
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


def _ctx(sdd, w, xi0, eta0, sub):
    import torch
    ny, nx = w.shape
    return sdd.sdd_init(nx, ny, sub, sub, w=torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda(),
                        xi0=torch.from_numpy(np.ascontiguousarray(xi0)).cuda(),
                        eta0=torch.from_numpy(np.ascontiguousarray(eta0)).cuda())


CASES = [
    # n, subdomains, w: 63^2 subdomains (6 levels), 31^2 (5 levels, ring with a 51:1 contrast), 127^2
    (129, 2, "front", 5e-3),
    (129, 4, "ring", 1e-3),
    (257, 2, "bump", 1e-2),
]


def _w(kind, n):
    if kind == "front":
        return W.w_front(n, 0.1)
    if kind == "ring":
        return W.w_ring(n, 0.0)
    return W.w_smooth_random(n, 8) * W.w_bump(n, 0.6, 0.4, 0.15, 4.0)


@pytest.mark.parametrize("n,sub,kind,Dt", CASES)
def test_multigrid_solve_matches_lu(sdd, oracle_mod, n, sub, kind, Dt):
    from oracle import solver
    import torch
    w = _w(kind, n).astype(np.float32).astype(np.float64)
    X, Y = W.grid(n)
    prev = [X + 0.03 * np.sin(2 * np.pi * X) * np.sin(np.pi * Y), Y + 0.02 * np.sin(np.pi * X)]
    ctx = _ctx(sdd, w, prev[0], prev[1], sub)
    sdd.sdd_set_solver(ctx, sdd.SDD_SOLVER_MG)
    assert sdd.sdd_solver_in_use(ctx) == 2
    ii, jj = W.interface_nodes(n, n, sub, sub)
    rng = np.random.default_rng(2)
    vx = X[jj, ii] + rng.normal(0, 1e-3, ii.size)
    ve = Y[jj, ii] + rng.normal(0, 1e-3, ii.size)
    gx, ge, iters = sdd.sdd_subdomain_solve(ctx, Dt, torch.from_numpy(vx).cuda(), torch.from_numpy(ve).cuda(),
                                            rtol=1e-12, max_iter=200)
    assert 0 < iters <= 30, iters
    faces = oracle_mod.winslow_faces(w)
    bx = oracle_mod.boundary_grid(faces, n, n, 0, prev[0])
    be = oracle_mod.boundary_grid(faces, n, n, 1, prev[1])
    bx[jj, ii] = vx
    be[jj, ii] = ve
    ox, oe = solver.subdomain_solve(w, prev, [bx, be], sub, sub, Dt)
    np.testing.assert_allclose(gx.cpu().numpy(), ox, rtol=0, atol=1e-9)
    np.testing.assert_allclose(ge.cpu().numpy(), oe, rtol=0, atol=1e-9)
    # far fewer iterations than the Jacobi preconditioner on the same systems
    sdd.sdd_set_solver(ctx, sdd.SDD_SOLVER_JACOBI)
    _, _, it_j = sdd.sdd_subdomain_solve(ctx, Dt, torch.from_numpy(vx).cuda(), torch.from_numpy(ve).cuda(),
                                         rtol=1e-12, max_iter=100000)
    assert it_j > 3 * iters, (it_j, iters)


def test_multigrid_mesh_steps_match_oracle(sdd, oracle_mod):
    # the GPU's trajectory and the oracle's (LU solves) from the same start, each on its own fields
    import torch
    from tests import _parity as PT
    n, sub, dt, Dt, paths = 129, 2, 1e-4, 1e-2, 2000
    xi, eta = W.identity_fields(n)
    ctx = _ctx(sdd, W.w_front(n, 0.0), xi, eta, sub)
    sdd.sdd_set_solver(ctx, sdd.SDD_SOLVER_MG)
    ii, jj = W.interface_nodes(n, n, sub, sub)
    state, gap = [xi, eta], 0.0
    for step in range(2):
        w = W.w_front(n, step * Dt)
        sdd.sdd_set_w(ctx, torch.from_numpy(w).cuda())
        sdd.sdd_step(ctx, dt=dt, Dt=Dt, seed=5, paths_per_node=paths, rtol=1e-12, max_iter=200)
        sdd.sdd_sync(ctx)
        g = {k: v.cpu().numpy() for k, v in sdd.sdd_last_interface_stats(ctx).items()}
        new, o = oracle_mod.dd_step(w, state[0], state[1], sub_x=sub, sub_y=sub, dt=dt, Dt=Dt, n_paths=paths,
                                    seed=5, step_index=step, nodes_ij=(ii, jj))
        gfields = [a.cpu().numpy() for a in sdd.sdd_get_fields(ctx)]
        gap = PT.assert_trajectory_step(g, o, gfields, new, gap, slack=1e-4, tag=f"step {step}")
        state = new


def test_multigrid_availability(sdd):
    # unequal subdomains (40 nodes in two halves) or even sizes do not coarsen
    for n, sub, auto in ((40, 2, 1), (34, 1, 1)):
        ctx = _ctx(sdd, np.ones((n, n)), *W.identity_fields(n), sub)
        with pytest.raises(sdd.SddError) as e:
            sdd.sdd_set_solver(ctx, sdd.SDD_SOLVER_MG)
        assert e.value.status == sdd.SDD_EINVAL
        assert sdd.sdd_solver_in_use(ctx) == auto
    # automatic: multigrid where the register-resident Jacobi kernel does not fit
    ctx = _ctx(sdd, np.ones((513, 513)), *W.identity_fields(513), 2)
    assert sdd.sdd_solver_in_use(ctx) == 2
    ctx = _ctx(sdd, np.ones((65, 65)), *W.identity_fields(65), 2)
    assert sdd.sdd_solver_in_use(ctx) == 1
    ctx = _ctx(sdd, np.ones((257, 257)), *W.identity_fields(257), 2)    # 127^2 unknowns per subdomain
    assert sdd.sdd_solver_in_use(ctx) == 2


def test_multigrid_nonconvergence_is_a_status(sdd):
    import torch
    n = 129
    ctx = _ctx(sdd, W.w_ring(n, 0.0), *W.identity_fields(n), 2)
    sdd.sdd_set_solver(ctx, sdd.SDD_SOLVER_MG)
    x, y = sdd.sdd_interface_nodes(ctx)
    v = torch.from_numpy(x + 0.01).cuda()
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_subdomain_solve(ctx, 1e-2, v, v, rtol=1e-14, max_iter=2)
    assert e.value.status == sdd.SDD_ENOCONV
