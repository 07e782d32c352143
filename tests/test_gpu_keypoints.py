"""Key points and interface fill on the GPU against the oracle (Sec. 4, Sec. 5).

The key-point decision is index work: the GPU's mask must equal the oracle's bit
for bit (both take the same double-precision differences of rho = 1 / w). The
fill must equal scipy's PCHIP through the same anchors."""
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


@pytest.fixture(scope="module")
def kp(oracle_mod):
    from oracle import keypoints
    return keypoints


def _ctx(sdd, w, xi0, eta0, sub):
    import torch
    ny, nx = w.shape
    return sdd.sdd_init(nx, ny, sub, sub, w=torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda(),
                        xi0=torch.from_numpy(np.ascontiguousarray(xi0)).cuda(),
                        eta0=torch.from_numpy(np.ascontiguousarray(eta0)).cuda())


def _bump_in_x(n, c, s):
    X, _ = W.grid(n)
    return 1.0 / (1.0 + 4.0 * np.exp(-((X - c) ** 2) / s ** 2))


MASKS = [(41, 2, lambda n: W.w_paper_ring(n, 0.0)), (41, 2, lambda n: W.w_paper_ring(n, 0.3)),
         (65, 2, lambda n: W.w_front(n, 0.2)), (129, 4, lambda n: _bump_in_x(n, 0.37, 0.08)),
         (129, 4, lambda n: W.w_ring(n, 0.1)), (257, 2, lambda n: W.w_smooth_random(n, 5)),
         (65, 3, lambda n: np.ones((n, n)))]


@pytest.mark.parametrize("n,sub,wf", MASKS)
def test_keypoint_mask_bit_exact(sdd, kp, n, sub, wf):
    w = np.asarray(wf(n), np.float32)
    ctx = _ctx(sdd, w, *W.identity_fields(n), sub)
    for spacing in (0, 7):
        sdd.sdd_set_keypoints(ctx, True, spacing)
        g = sdd.sdd_keypoint_mask(ctx).cpu().numpy().astype(bool)
        o = kp.key_mask(w.astype(np.float64), sub, sub, spacing)
        np.testing.assert_array_equal(g, o)


def test_keypoint_steps_match_oracle(sdd, kp, oracle_mod):
    # the GPU's trajectory with key points and the oracle's from the same start, each on its own
    # fields: the key points' estimates within the trajectory bound (3 SE plus the previous
    # fields' gap)
    import torch
    n, sub, dt, Dt, paths = 41, 2, 5e-5, 1e-3, 4000
    xi, eta = W.identity_fields(n)
    ctx = _ctx(sdd, W.w_paper_ring(n, 0.0), xi, eta, sub)
    sdd.sdd_set_keypoints(ctx, True, 8)
    ii, jj = W.interface_nodes(n, n, sub, sub)
    state, gap = [xi, eta], 0.0
    for step in range(3):
        w = W.w_paper_ring(n, step * Dt)
        sdd.sdd_set_w(ctx, torch.from_numpy(w).cuda())
        sdd.sdd_step(ctx, dt=dt, Dt=Dt, seed=4, paths_per_node=paths, rtol=1e-13, max_iter=50000)
        sdd.sdd_sync(ctx)
        g = {k: v.cpu().numpy() for k, v in sdd.sdd_last_interface_stats(ctx).items()}
        new, o = oracle_mod.dd_step(w, state[0], state[1], sub_x=sub, sub_y=sub, dt=dt, Dt=Dt, n_paths=paths,
                                    seed=4, step_index=step, nodes_ij=(ii, jj), keypoints=True, key_spacing=8)
        m = o["key"]
        assert 0 < m.sum() < m.size
        np.testing.assert_array_equal(g["path_steps"] > 0, m)          # paths ran exactly at the key points
        for f in ("xi", "eta"):
            d = np.abs(g["mean_" + f][m] - o["mean_" + f][m])
            assert np.all(d <= 3 * o["se_" + f][m] + gap + 1e-4), (step, f, d.max())
        # the filled nodes follow PCHIP, whose derivative limiter is not continuous in the data,
        # so their gap has no bound from the key points' (the fill itself is checked on seeded
        # values below); the solve's maximum principle still bounds the new fields' gap by the
        # larger of all interface values' gap and the previous fields'
        iface = max(float(np.abs(g["mean_xi"] - o["mean_xi"]).max()), float(np.abs(g["mean_eta"] - o["mean_eta"]).max()))
        gfields = [a.cpu().numpy() for a in sdd.sdd_get_fields(ctx)]
        new_gap = max(float(np.abs(gfields[0] - new[0]).max()), float(np.abs(gfields[1] - new[1]).max()))
        assert new_gap <= max(iface, gap) + 1e-9, (step, new_gap, iface, gap)
        gap = new_gap
        state = new


def _fill_case(n, sub, seed):
    """Seeded interface values and a key mask (crossings always key) for the fill checks."""
    ii, jj = W.interface_nodes(n, n, sub, sub)
    rng = np.random.default_rng(seed)
    vx = ii / (n - 1) + 0.01 * rng.standard_normal(ii.size)
    ve = jj / (n - 1) + 0.01 * rng.standard_normal(ii.size)
    lines = set(W.interface_lines(n, sub))
    cross = np.array([(i in lines) and (j in lines) for i, j in zip(ii, jj)])
    mask = cross | (rng.random(ii.size) < 0.25)
    return vx, ve, mask


@pytest.mark.parametrize("n,sub", [(41, 2), (65, 3), (129, 4)])
def test_fill_on_seeded_values_is_pchip(sdd, kp, oracle_mod, n, sub):
    import torch
    w = W.w_paper_ring(n, 0.1)
    ctx = _ctx(sdd, w, *W.identity_fields(n), sub)
    vx, ve, mask = _fill_case(n, sub, n + sub)
    gx, ge = sdd.sdd_keypoint_fill(ctx, torch.from_numpy(mask.astype(np.uint8)).cuda(), torch.from_numpy(vx).cuda(),
                                   torch.from_numpy(ve).cuda())
    faces = oracle_mod.winslow_faces(w.astype(np.float64))
    fx, fe = kp.pchip_fill(vx, ve, mask, faces, n, n, sub, sub)
    np.testing.assert_allclose(gx.cpu().numpy(), fx, rtol=0, atol=1e-10)
    np.testing.assert_allclose(ge.cpu().numpy(), fe, rtol=0, atol=1e-10)
    np.testing.assert_array_equal(gx.cpu().numpy()[mask], vx[mask])      # the key values stay


def test_fill_on_lines_too_long_for_shared_memory(sdd, kp, oracle_mod):
    """Lines of 3401 positions: the fill's staging (61 bytes a position) exceeds the
    shared memory it may take, so the fill runs with its anchors in global scratch;
    it must still be scipy's PCHIP through the given key values (seeded), and the
    key points of a mesh step must be where the paths ran."""
    import torch
    n, sub = 3401, 2
    w = W.w_paper_ring(n, 0.0)
    ctx = _ctx(sdd, w, *W.identity_fields(n), sub)
    vx, ve, mask = _fill_case(n, sub, 11)
    gx, ge = sdd.sdd_keypoint_fill(ctx, torch.from_numpy(mask.astype(np.uint8)).cuda(), torch.from_numpy(vx).cuda(),
                                   torch.from_numpy(ve).cuda())
    faces = oracle_mod.winslow_faces(w.astype(np.float64))
    fx, fe = kp.pchip_fill(vx, ve, mask, faces, n, n, sub, sub)
    np.testing.assert_allclose(gx.cpu().numpy(), fx, rtol=0, atol=1e-10)
    np.testing.assert_allclose(ge.cpu().numpy(), fe, rtol=0, atol=1e-10)
    sdd.sdd_set_keypoints(ctx, True, 8)
    sdd.sdd_set_w(ctx, torch.from_numpy(w).cuda())
    sdd.sdd_step(ctx, dt=5e-5, Dt=1e-3, seed=2, paths_per_node=200)
    sdd.sdd_sync(ctx)
    g = {k: v.cpu().numpy() for k, v in sdd.sdd_last_interface_stats(ctx).items()}
    m = sdd.sdd_keypoint_mask(ctx).cpu().numpy().astype(bool)
    assert 0 < m.sum() < m.size
    np.testing.assert_array_equal(g["path_steps"] > 0, m)
