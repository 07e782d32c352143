"""Direct subdomain solves (banded Cholesky, the paper's direct solve for small
subdomains) against the oracle's sparse LU, and their place among the solvers."""
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


def _ctx(sdd, w, xi0, eta0, sub_x, sub_y):
    import torch
    ny, nx = w.shape
    return sdd.sdd_init(nx, ny, sub_x, sub_y, w=torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda(),
                        xi0=torch.from_numpy(np.ascontiguousarray(xi0)).cuda(),
                        eta0=torch.from_numpy(np.ascontiguousarray(eta0)).cuda())


def _grid(nx, ny):
    x = np.linspace(0.0, 1.0, nx)
    y = np.linspace(0.0, 1.0, ny)
    return np.meshgrid(x, y)


@pytest.mark.parametrize("nx,ny,sub_x,sub_y,Dt", [(41, 41, 2, 2, 5e-3),    # ring41's 19 x 19 subdomains
                                                  (40, 40, 2, 2, 1e-2),    # 19 and 18 rows and columns
                                                  (41, 33, 2, 2, 2e-3),    # 19 x 15
                                                  (65, 65, 4, 4, 1e-1),    # 15 x 15, sixteen subdomains
                                                  (17, 65, 1, 2, 5e-3)])   # 15 columns x 31 rows
def test_direct_solve_matches_lu(sdd, oracle_mod, nx, ny, sub_x, sub_y, Dt):
    from oracle import solver
    import torch
    X, Y = _grid(nx, ny)
    w = (1.0 + 3.0 * np.exp(-((X - 0.6) ** 2 + (Y - 0.4) ** 2) / 0.15 ** 2)).astype(np.float32).astype(np.float64)
    prev = [X + 0.03 * np.sin(2 * np.pi * X) * np.sin(np.pi * Y), Y + 0.02 * np.sin(np.pi * X)]
    ctx = _ctx(sdd, w, prev[0], prev[1], sub_x, sub_y)
    sdd.sdd_set_solver(ctx, sdd.SDD_SOLVER_DIRECT)
    assert sdd.sdd_solver_in_use(ctx) == 3
    ii, jj = W.interface_nodes(nx, ny, sub_x, sub_y)
    rng = np.random.default_rng(5)
    vx = X[jj, ii] + rng.normal(0, 1e-3, ii.size)
    ve = Y[jj, ii] + rng.normal(0, 1e-3, ii.size)
    gx, ge, iters = sdd.sdd_subdomain_solve(ctx, Dt, torch.from_numpy(vx).cuda(), torch.from_numpy(ve).cuda(),
                                            rtol=1e-13, max_iter=100)
    assert iters == 1
    faces = oracle_mod.winslow_faces(w)
    bx = oracle_mod.boundary_grid(faces, nx, ny, 0, prev[0])
    be = oracle_mod.boundary_grid(faces, nx, ny, 1, prev[1])
    bx[jj, ii] = vx
    be[jj, ii] = ve
    ox, oe = solver.subdomain_solve(w, prev, [bx, be], sub_x, sub_y, Dt)
    np.testing.assert_allclose(gx.cpu().numpy(), ox, rtol=0, atol=1e-12)
    np.testing.assert_allclose(ge.cpu().numpy(), oe, rtol=0, atol=1e-12)


def test_direct_solve_availability_and_choice(sdd):
    def ctx(n, sub):
        return _ctx(sdd, np.ones((n, n)), *W.identity_fields(n), sub, sub)
    # never the automatic choice (Jacobi-PCG is faster where the direct solve fits)
    assert sdd.sdd_solver_in_use(ctx(41, 2)) == 1
    assert sdd.sdd_solver_in_use(ctx(257, 2)) == 2
    for n in (41, 65):                                   # 19 x 19 and 31 x 31 fit
        c = ctx(n, 2)
        sdd.sdd_set_solver(c, sdd.SDD_SOLVER_DIRECT)
        assert sdd.sdd_solver_in_use(c) == 3
    for n in (69, 257):                                  # 33 columns: wider than a warp's band
        c = ctx(n, 2)
        with pytest.raises(sdd.SddError) as e:
            sdd.sdd_set_solver(c, sdd.SDD_SOLVER_DIRECT)
        assert e.value.status == sdd.SDD_EINVAL


def test_direct_residual_check_reports_a_missed_tolerance(sdd):
    import torch
    n = 41
    c = _ctx(sdd, W.w_smooth_random(n, 2), *W.identity_fields(n), 2, 2)
    sdd.sdd_set_solver(c, sdd.SDD_SOLVER_DIRECT)
    x, y = sdd.sdd_interface_nodes(c)
    v = torch.from_numpy(x + 0.01).cuda()
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_subdomain_solve(c, 1e-2, v, v, rtol=0.0, max_iter=10)   # no rounded residual is exactly zero
    assert e.value.status == sdd.SDD_ENOCONV


def test_direct_mesh_steps_match_jacobi(sdd):
    """The Sec. 5 experiment's mesh steps (pipelined, key points) with the direct
    solve and with Jacobi-PCG refined to 1e-13: the same fields."""
    import torch
    n = 41
    out = []
    for solver in (sdd.SDD_SOLVER_DIRECT, sdd.SDD_SOLVER_JACOBI):
        c = _ctx(sdd, W.w_paper_ring(n, 0.0), *W.identity_fields(n), 2, 2)
        sdd.sdd_set_solver(c, solver)
        sdd.sdd_set_keypoints(c, True, 8)
        for k in range(6):
            sdd.sdd_set_w(c, torch.from_numpy(W.w_paper_ring(n, k * 1e-3)).cuda())
            sdd.sdd_step(c, dt=5e-5, Dt=1e-3, seed=3, paths_per_node=2000, rtol=1e-13, max_iter=50000)
        assert sdd.sdd_pipeline_in_use(c)
        out.append([t.cpu().numpy() for t in sdd.sdd_get_fields(c)])
        sdd.sdd_sync(c)
    np.testing.assert_allclose(out[0][0], out[1][0], rtol=0, atol=1e-9)
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=0, atol=1e-9)
