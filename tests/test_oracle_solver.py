"""Pins of the oracle's implicit subdomain solve (Sec. 4, reading R14)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import solver


def test_linear_field_is_stationary():
    # w = w(y) and xi = x: every x-flux is equal and every y-difference is zero
    n = 21
    X, Y = W.grid(n)
    w = 1.0 + 3.0 * np.exp(-((Y - 0.4) / 0.2) ** 2)
    out = solver.subdomain_solve(w, [X, Y * 0 + 0.3], [X, Y * 0 + 0.3], 2, 2, 1e-2)
    np.testing.assert_allclose(out[0], X, atol=1e-13)
    np.testing.assert_allclose(out[1], 0.3, atol=1e-13)


def test_one_dimensional_steady_state_is_stationary(oracle_mod):
    # w = w(x): the cumulative trapezoid of w has constant discrete flux
    # (xi_{i+1} - xi_i) / wbar_{i+1/2}, so it is an exact discrete steady state
    n = 33
    X, Y = W.grid(n)
    w = 1.0 + 5.0 * np.exp(-((X - 0.3) / 0.1) ** 2)
    seg = oracle_mod.split_faces(oracle_mod.winslow_faces(w), n, n)
    xi = np.tile(seg[(0, 2)], (n, 1))
    out = solver.subdomain_solve(w, [xi, Y], [xi, Y], 3, 2, 5e-3)
    np.testing.assert_allclose(out[0], xi, atol=1e-13)
    np.testing.assert_allclose(out[1], Y, atol=1e-13)


def test_matrix_is_symmetric_m_matrix():
    n = 12
    w = W.w_smooth_random(n, 4).astype(np.float64)
    A = solver.dense_matrix(w, 1, n - 1, 1, n - 1, 3e-3)
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-9 * np.abs(A).max())
    off = A - np.diag(np.diag(A))
    assert np.all(off <= 0)
    assert np.all(np.diag(A) > -off.sum(axis=1))          # strictly diagonally dominant
    assert np.linalg.eigvalsh(A).min() > 0


def test_maximum_principle():
    # an M-matrix step keeps the new field between the extremes of the data
    n = 25
    rng = np.random.default_rng(0)
    w = W.w_smooth_random(n, 2).astype(np.float64)
    prev = rng.uniform(0.2, 0.7, size=(n, n))
    bnd = rng.uniform(0.1, 0.9, size=(n, n))
    out = solver.subdomain_solve(w, [prev], [bnd], 2, 2, 1e-2)[0]
    assert out.min() >= 0.1 - 1e-12 and out.max() <= 0.9 + 1e-12


def test_decomposed_solve_matches_global_solve():
    # interface values taken from the global solution make the subdomain
    # solves reproduce it (the systems decouple exactly along the interfaces)
    n = 29
    X, Y = W.grid(n)
    w = W.w_smooth_random(n, 9).astype(np.float64)
    prev = [X + 0.1 * np.sin(3 * Y), Y + 0.05 * np.sin(2 * X)]
    g = solver.global_solve(w, prev, prev, 4e-3)
    out = solver.subdomain_solve(w, prev, g, 2, 3, 4e-3)
    for a, b in zip(out, g):
        np.testing.assert_allclose(a, b, atol=1e-12)


def test_heat_equation_converges():
    # w = 1: one mode decays by exp(-2 pi^2 t); error O(h^2 + Delta t)
    errs = []
    for n, Dt in ((17, 2e-3), (33, 5e-4)):
        X, Y = W.grid(n)
        u = np.sin(np.pi * X) * np.sin(np.pi * Y)
        w = np.ones((n, n))
        t = 0.0
        while t < 0.02 - 1e-12:
            u = solver.global_solve(w, [u], [u * 0], Dt)[0]
            t += Dt
        exact = math.exp(-2 * math.pi ** 2 * 0.02) * np.sin(np.pi * X) * np.sin(np.pi * Y)
        errs.append(np.abs(u - exact).max())
    assert errs[1] < errs[0] / 3.0, errs
    assert errs[1] < 5e-3


def test_symmetrised_form_agrees_with_direct_discretisation():
    # reading R14: the symmetrised implicit step and a direct central
    # discretisation of Eq. (3) differ by O(h^2)
    diffs = []
    for n in (17, 33):
        X, Y = W.grid(n)
        w = 1.0 + 2.0 * np.exp(-((X - 0.5) ** 2 + (Y - 0.4) ** 2) / 0.08)
        prev = np.sin(np.pi * X) * np.sin(np.pi * Y) + X
        bnd = X.copy()
        a = solver.global_solve(w, [prev], [bnd], 1e-3)[0]
        b = solver.nonconservative_step(w, prev, bnd, 1e-3)
        diffs.append(np.abs(a - b).max())
    assert diffs[1] < diffs[0] / 3.0, diffs
