"""The paper's Sec. 5 experiment end to end on the GPU.

w = 1 / rho with rho = 1 + 10 exp(-50 |(x - 1/2 - cos(2 pi t)/4)^2 + (y - 1/2 - sin(2 pi t)/4)^2 - 1/100|),
41 x 41 nodes, four subdomains, Delta t = 1e-3 up to t = 0.75 (750 mesh steps), 20 sub-steps per step,
1e4 paths per interface node, from the uniform mesh. The paper shows the meshes at t = 0.25, 0.5, 0.75
and reports smooth, adapting meshes. Checked here: no mesh cell folds (every cell of the computational
coordinates keeps its orientation) and the fields stay close to the same implicit scheme solved on the
whole square without decomposition (the oracle's sparse LU), within the Monte Carlo error the interface
values carry; and the mesh does adapt (it moves away from the uniform mesh towards the ring).
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


def folded_cells(xi, eta):
    """Cells whose image quadrilateral in (xi, eta) is not positively oriented at every corner."""
    p = np.stack([xi, eta], axis=-1)
    c00, c10, c11, c01 = p[:-1, :-1], p[:-1, 1:], p[1:, 1:], p[1:, :-1]
    quad = [c00, c10, c11, c01]
    bad = np.zeros(xi[:-1, :-1].shape, dtype=bool)
    for k in range(4):
        a, b, c = quad[k - 1], quad[k], quad[(k + 1) % 4]
        e1, e2 = b - a, c - b
        bad |= (e1[..., 0] * e2[..., 1] - e1[..., 1] * e2[..., 0]) <= 0
    return int(bad.sum())


@pytest.mark.parametrize("keypoints", [True, False])
def test_sec5_moving_ring_mesh(sdd, oracle_mod, keypoints):
    # keypoints=True is the paper's setup (estimates at the key points, PCHIP elsewhere), with a key
    # point also at every 8th node of each line
    import torch
    from oracle import solver
    n, Dt, K, paths, steps = 41, 1e-3, 20, 10000, 750
    xi0, eta0 = W.identity_fields(n)
    ctx = sdd.sdd_init(n, n, 2, 2, w=torch.from_numpy(W.w_paper_ring(n, 0.0)).cuda(),
                       xi0=torch.from_numpy(xi0).cuda(), eta0=torch.from_numpy(eta0).cuda())
    sdd.sdd_set_keypoints(ctx, keypoints, 8)
    ref = [xi0.copy(), eta0.copy()]
    snaps = {}
    for k in range(steps):
        w = W.w_paper_ring(n, k * Dt)
        sdd.sdd_set_w(ctx, torch.from_numpy(w).cuda())
        sdd.sdd_step(ctx, dt=Dt / K, Dt=Dt, seed=0, paths_per_node=paths, rtol=1e-12, max_iter=20000)
        faces = oracle_mod.winslow_faces(w.astype(np.float64))
        bx = oracle_mod.boundary_grid(faces, n, n, 0, ref[0])
        be = oracle_mod.boundary_grid(faces, n, n, 1, ref[1])
        ref = solver.global_solve(w, ref, [bx, be], Dt)
        if k + 1 in (250, 500, 750):
            gx, ge = (a.cpu().numpy() for a in sdd.sdd_get_fields(ctx))
            snaps[k + 1] = (gx, ge, ref[0].copy(), ref[1].copy())
    sdd.sdd_sync(ctx)
    X, Y = W.grid(n)
    report = {}
    for k, (gx, ge, rx, re) in snaps.items():
        dev = max(np.abs(gx - rx).max(), np.abs(ge - re).max())
        moved = max(np.abs(gx - X).max(), np.abs(ge - Y).max())
        report[k] = (folded_cells(gx, ge), folded_cells(rx, re), dev, moved)
    print(keypoints, report)
    for k, (fg, fr, dev, moved) in report.items():
        assert fg == 0 and fr == 0, (k, fg, fr)
        # the interface values carry the Monte Carlo error and the plain exit test's sqrt(dt) bias
        # (Sec. 4), and with key points the fill's interpolation error: the mesh stays within half a
        # cell (h / 2 = 0.0125) of the deterministic scheme, one cell with key points
        assert dev < (0.025 if keypoints else 0.0125), (k, dev)
        assert moved > 0.1, (k, moved)      # while it moves by several cells towards the ring
