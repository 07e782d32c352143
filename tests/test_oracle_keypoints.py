"""Pins of the oracle's key-point placement and PCHIP fill (Sec. 4, Sec. 5)."""
import math

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def kp(oracle_mod):
    from oracle import keypoints
    return keypoints


def _bump_in_x(n, c, s, a=4.0):
    X, _ = W.grid(n)
    return 1.0 / (1.0 + a * np.exp(-((X - c) ** 2) / s ** 2))


def test_node_list_matches_the_estimators_order(kp):
    for n, sub in ((65, 2), (41, 2), (42, 3), (129, 4)):
        ii, jj = W.interface_nodes(n, n, sub, sub)
        assert kp.node_list(n, n, sub, sub) == list(zip(ii.tolist(), jj.tolist()))


def test_key_points_sit_at_the_analytic_extrema(kp):
    # rho = 1 + a exp(-(x - c)^2 / s^2) along x only: rho_x has its extrema at c -+ s / sqrt(2), rho_xx at
    # c and c -+ s sqrt(3/2); on the vertical lines rho does not change, so only the crossings are key
    n, c, s = 129, 0.37, 0.08
    w = _bump_in_x(n, c, s)
    mask = kp.key_mask(w, 2, 2)
    nodes = kp.node_list(n, n, 2, 2)
    J = kp.line_indices(n, 2)[0]
    I = kp.line_indices(n, 2)[0]
    key_h = sorted(i for (i, j), m in zip(nodes, mask) if m and j == J and i != I)
    want = [c - s * math.sqrt(1.5), c - s / math.sqrt(2), c, c + s / math.sqrt(2), c + s * math.sqrt(1.5)]
    assert len(key_h) == len(want), key_h
    for i, x in zip(key_h, want):
        assert abs(i / (n - 1) - x) <= 1.0 / (n - 1), (i, x)
    key_v = [(i, j) for (i, j), m in zip(nodes, mask) if m and i == I]
    assert key_v == [(I, J)]


def test_flat_density_keeps_only_the_crossings(kp):
    mask = kp.key_mask(np.ones((65, 65)), 4, 4)
    nodes = kp.node_list(65, 65, 4, 4)
    vi, hj = set(kp.line_indices(65, 4)), set(kp.line_indices(65, 4))
    assert [nodes[k] for k in np.flatnonzero(mask)] == [(i, j) for (i, j) in nodes if i in vi and j in hj]


def test_pchip_fill_properties(kp, oracle_mod):
    n, sub = 65, 2
    w = W.w_front(n, 0.2)
    faces = oracle_mod.winslow_faces(w.astype(np.float64))
    mask = kp.key_mask(w, sub, sub)
    nodes = kp.node_list(n, n, sub, sub)
    # the face data of xi, eta along the lines' ends, and values that are linear in the line coordinate
    # between them, are reproduced exactly; key values are kept
    X, Y = W.grid(n)
    F = oracle_mod.split_faces(faces, n, n)
    vx = np.zeros(len(nodes))
    ve = np.zeros(len(nodes))
    lines = kp.lines(n, n, sub, sub)
    for orient, fixed, pts in lines:
        for t in range(1, n - 1):
            i, j = pts[t]
            k = nodes.index((i, j))
            if orient == "v":
                a0, a1 = F[(0, 2)][fixed], F[(0, 3)][fixed]
                b0, b1 = F[(1, 2)][fixed], F[(1, 3)][fixed]
            else:
                if (i, j) in nodes[: (n - 2) * len(kp.line_indices(n, sub))]:
                    continue
                a0, a1 = F[(0, 0)][fixed], F[(0, 1)][fixed]
                b0, b1 = F[(1, 0)][fixed], F[(1, 1)][fixed]
            vx[k] = a0 + (a1 - a0) * t / (n - 1)
            ve[k] = b0 + (b1 - b0) * t / (n - 1)
    fx, fe = kp.pchip_fill(np.where(mask, vx, np.nan), np.where(mask, ve, np.nan), mask, faces, n, n, sub, sub)
    # the crossing belongs to the vertical line's linear profile; horizontal lines through it are not
    # linear there in general, so compare the vertical lines only
    nv = (n - 2) * len(kp.line_indices(n, sub))
    np.testing.assert_allclose(fx[:nv], vx[:nv], atol=1e-12)
    np.testing.assert_allclose(fe[:nv], ve[:nv], atol=1e-12)
    np.testing.assert_array_equal(fx[mask], vx[mask])
    # monotone anchors give a monotone fill (PCHIP preserves monotonicity)
    assert np.all(np.isfinite(fx)) and np.all(np.isfinite(fe))


def test_keypoint_step_uses_fewer_nodes_and_stays_close(oracle_mod, kp):
    # the Sec. 5 density on 41 x 41: the key-point step estimates at a fraction of the nodes and its
    # fields stay close to the all-node step (same streams at the key nodes)
    n, sub = 41, 2
    w = W.w_paper_ring(n, 0.0)
    xi, eta = W.identity_fields(n)
    ii, jj = W.interface_nodes(n, n, sub, sub)
    kw = dict(sub_x=sub, sub_y=sub, dt=5e-5, Dt=1e-3, n_paths=2000, seed=3, step_index=0, nodes_ij=(ii, jj))
    full, rf = oracle_mod.dd_step(w, xi, eta, **kw)
    key, rk = oracle_mod.dd_step(w, xi, eta, keypoints=True, **kw)
    m = rk["key"]
    assert 0 < m.sum() < 0.5 * m.size
    np.testing.assert_array_equal(rk["mean_xi"][m], rf["mean_xi"][m])
    assert np.all(rk["path_steps"][~m] == 0)
    gap = max(np.abs(key[0] - full[0]).max(), np.abs(key[1] - full[1]).max())
    assert gap < 5e-3, gap


def test_spacing_adds_every_gth_position(kp):
    n, sub, g = 41, 2, 8
    w = W.w_paper_ring(n, 0.0)
    base = kp.key_mask(w, sub, sub)
    spaced = kp.key_mask(w, sub, sub, g)
    assert np.all(spaced >= base)
    nodes = kp.node_list(n, n, sub, sub)
    I = kp.line_indices(n, sub)[0]
    for k, (i, j) in enumerate(nodes):
        t = j if i == I else i
        if t % g == 0:
            assert spaced[k], (i, j)
        elif not base[k]:
            assert not spaced[k], (i, j)
