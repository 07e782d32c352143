"""Pins of the oracle's grid operations: finite-difference drift, bilinear
interpolation and the 1D Winslow face data, each against a closed form."""
import math

import numpy as np
import pytest

import workloads as W


def test_drift_exact_for_quadratic_w(oracle_mod):
    # central and one-sided second-order differences are exact on quadratics,
    # so b = -grad w / w holds to rounding at every node, edges included (R4)
    X, Y = W.grid(9, 7)
    w = 1.0 + 0.3 * X ** 2 + 0.2 * Y ** 2 + 0.1 * X * Y + 0.5 * X - 0.25 * Y
    bx, by = oracle_mod.drift_field(w)
    wx = 0.6 * X + 0.1 * Y + 0.5
    wy = 0.4 * Y + 0.1 * X - 0.25
    np.testing.assert_allclose(bx, -wx / w, rtol=0, atol=1e-12)
    np.testing.assert_allclose(by, -wy / w, rtol=0, atol=1e-12)


def test_drift_second_order(oracle_mod):
    errs = []
    for n in (17, 33, 65):
        X, Y = W.grid(n)
        w = np.exp(np.sin(2 * X) + 0.5 * np.cos(3 * Y))
        bx, by = oracle_mod.drift_field(w)
        ex = -2 * np.cos(2 * X)
        ey = 1.5 * np.sin(3 * Y)
        errs.append(max(np.abs(bx - ex).max(), np.abs(by - ey).max()))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.6 and 3.5 < r2 < 4.6, errs


def test_constant_w_has_zero_drift(oracle_mod):
    bx, by = oracle_mod.drift_field(np.full((5, 6), 3.7))
    assert np.abs(bx).max() < 1e-14 and np.abs(by).max() < 1e-14


def test_bilinear_reproduces_bilinear_functions(oracle_mod):
    X, Y = W.grid(11, 6)
    a, b, c, d = 0.3, -1.2, 2.5, 0.7
    f = a + b * X + c * Y + d * X * Y
    rng = np.random.default_rng(0)
    for x, y in rng.uniform(0, 1, size=(200, 2)):
        assert oracle_mod.bilinear(f, x, y) == pytest.approx(a + b * x + c * y + d * x * y, abs=1e-13)
    for x, y in ((0, 0), (1, 1), (1, 0), (0, 1), (1.0, 0.37), (0.42, 1.0)):
        assert oracle_mod.bilinear(f, x, y) == pytest.approx(a + b * x + c * y + d * x * y, abs=1e-13)


def test_bilinear_hits_node_values(oracle_mod):
    rng = np.random.default_rng(3)
    f = rng.normal(size=(5, 7))
    for j in range(5):
        for i in range(7):
            assert oracle_mod.bilinear(f, i / 6, j / 4) == pytest.approx(f[j, i], abs=1e-14)


def test_bilinear_is_not_tensor_transposed(oracle_mod):
    # f depends on x only: f[j, i] = i; a transposed index would read j
    f = np.tile(np.arange(7, dtype=float), (4, 1))
    assert oracle_mod.bilinear(f, 0.5, 0.1) == pytest.approx(3.0)


def test_winslow_faces_linear_w(oracle_mod):
    # w = 1 + x + 2y is linear along every face: the trapezoid rule is exact
    nx, ny = 9, 5
    X, Y = W.grid(nx, ny)
    w = 1.0 + X + 2.0 * Y
    faces = oracle_mod.split_faces(oracle_mod.winslow_faces(w), nx, ny)
    x = np.arange(nx) / (nx - 1)
    y = np.arange(ny) / (ny - 1)
    np.testing.assert_allclose(faces[(0, 0)], 0.0)                                      # xi, x = 0
    np.testing.assert_allclose(faces[(0, 1)], 1.0)                                      # xi, x = 1
    np.testing.assert_allclose(faces[(0, 2)], (x + x ** 2 / 2) / 1.5, atol=1e-14)       # xi, y = 0
    np.testing.assert_allclose(faces[(0, 3)], (3 * x + x ** 2 / 2) / 3.5, atol=1e-14)   # xi, y = 1
    np.testing.assert_allclose(faces[(1, 0)], (y + y ** 2) / 2.0, atol=1e-14)           # eta, x = 0
    np.testing.assert_allclose(faces[(1, 1)], (2 * y + y ** 2) / 3.0, atol=1e-14)       # eta, x = 1
    np.testing.assert_allclose(faces[(1, 2)], 0.0)                                      # eta, y = 0
    np.testing.assert_allclose(faces[(1, 3)], 1.0)                                      # eta, y = 1


def test_winslow_faces_solve_1d_winslow(oracle_mod):
    # the face data satisfy the discrete 1D form of Eq. (2): constant flux (xi_{k+1} - xi_k) / wbar
    nx = ny = 33
    X, Y = W.grid(nx)
    w = 1 + 3 * np.exp(-((X - 0.4) ** 2 + (Y - 0.6) ** 2) / 0.05)
    faces = oracle_mod.split_faces(oracle_mod.winslow_faces(w), nx, ny)
    for seg, v in ((faces[(0, 2)], w[0, :]), (faces[(0, 3)], w[-1, :]), (faces[(1, 0)], w[:, 0]),
                   (faces[(1, 1)], w[:, -1])):
        flux = np.diff(seg) / (0.5 * (v[1:] + v[:-1]))
        np.testing.assert_allclose(flux, flux[0], rtol=1e-12)
        assert seg[0] == 0.0 and seg[-1] == pytest.approx(1.0, abs=1e-15)


def test_face_value_interpolates(oracle_mod):
    nx, ny = 5, 9
    faces = np.arange(oracle_mod.faces_len(nx, ny), dtype=float) ** 1.5
    seg = oracle_mod.split_faces(faces, nx, ny)
    for field in (0, 1):
        for face in range(4):
            v = seg[(field, face)]
            n = v.size
            for s in (0.0, 1.0, 0.3, 0.77):
                g = s * (n - 1)
                k = min(int(math.floor(g)), n - 2)
                want = v[k] + (g - k) * (v[k + 1] - v[k])
                assert oracle_mod.face_value(faces, nx, ny, field, face, s) == pytest.approx(want, rel=1e-14)
