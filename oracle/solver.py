"""Implicit finite-difference subdomain solve (Sec. 4, "Deterministic single-domain solver").

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper solves an implicit finite-difference discretisation of Eq. (3) on
each subdomain, with the interface values as Dirichlet data, by LU
factorisation, and gives no stencil. Reading R14: since

    -(1/w) grad w . grad xi + lap xi = w div((1/w) grad xi),

implicit Euler multiplied through by 1/w reads, at an unknown node (i, j),

    (xi_ij - xi^{n-1}_ij) / (w_ij Delta t)
        = sum over the four neighbours nb of (xi_nb - xi_ij) / (wbar h^2),

with wbar = (w_ij + w_nb) / 2 the face average and h the spacing in that
direction. The matrix is symmetric positive definite. The solve here is a
sparse LU factorisation (scipy's SuperLU), as in the paper.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _lines(n: int, parts: int):
    return [0] + [int(round(k * (n - 1) / parts)) for k in range(1, parts)] + [n - 1]


def subdomain_blocks(nx: int, ny: int, sub_x: int, sub_y: int):
    """Index ranges [i0, i1) x [j0, j1) of each subdomain's unknown nodes, row-major over subdomains."""
    xs = _lines(nx, sub_x)
    ys = _lines(ny, sub_y)
    out = []
    for b in range(sub_y):
        for a in range(sub_x):
            out.append((xs[a] + 1, xs[a + 1], ys[b] + 1, ys[b + 1]))
    return out


def assemble(w, prev, bc, i0, i1, j0, j1, Dt):
    """Matrix and right-hand sides (one per field) of one block of unknowns.

    w: (ny, nx) FP64 density at t_{n-1}; prev: list of (ny, nx) fields at
    t_{n-1}; bc: list of (ny, nx) arrays holding the Dirichlet values on the
    block's boundary ring. Returns (A (csc), [rhs per field]).
    """
    ny, nx = w.shape
    hx = 1.0 / (nx - 1)
    hy = 1.0 / (ny - 1)
    mx, my = i1 - i0, j1 - j0
    m = mx * my
    rows, cols, vals = [], [], []
    rhs = [np.zeros(m) for _ in prev]

    def idx(i, j):
        return (j - j0) * mx + (i - i0)

    for j in range(j0, j1):
        for i in range(i0, i1):
            r = idx(i, j)
            diag = 1.0 / (w[j, i] * Dt)
            for f, p in enumerate(prev):
                rhs[f][r] += p[j, i] / (w[j, i] * Dt)
            for (di, dj, h) in ((-1, 0, hx), (1, 0, hx), (0, -1, hy), (0, 1, hy)):
                ii, jj = i + di, j + dj
                c = 1.0 / (0.5 * (w[j, i] + w[jj, ii]) * h * h)
                diag += c
                if i0 <= ii < i1 and j0 <= jj < j1:
                    rows.append(r)
                    cols.append(idx(ii, jj))
                    vals.append(-c)
                else:
                    for f, b in enumerate(bc):
                        rhs[f][r] += c * b[jj, ii]
            rows.append(r)
            cols.append(r)
            vals.append(diag)
    A = sp.csc_matrix((vals, (rows, cols)), shape=(m, m))
    return A, rhs


def subdomain_solve(w, prev_fields, new_boundary, sub_x, sub_y, Dt):
    """One implicit step on every subdomain; interfaces and the outer boundary are Dirichlet.

    prev_fields: [xi^{n-1}, eta^{n-1}]; new_boundary: [xi, eta] grids whose
    boundary and interface-line entries hold the Dirichlet values at t_n
    (other entries are ignored). Returns the new [xi^n, eta^n].
    """
    w = np.asarray(w, dtype=np.float64)
    ny, nx = w.shape
    out = [np.array(b, dtype=np.float64, copy=True) for b in new_boundary]
    for (i0, i1, j0, j1) in subdomain_blocks(nx, ny, sub_x, sub_y):
        if i1 <= i0 or j1 <= j0:
            continue
        A, rhs = assemble(w, prev_fields, new_boundary, i0, i1, j0, j1, Dt)
        lu = spla.splu(A)
        for f in range(len(out)):
            out[f][j0:j1, i0:i1] = lu.solve(rhs[f]).reshape(j1 - j0, i1 - i0)
    return out


def global_solve(w, prev_fields, boundary, Dt):
    """The same implicit step on the whole square (no decomposition): only the outer boundary is Dirichlet."""
    w = np.asarray(w, dtype=np.float64)
    ny, nx = w.shape
    out = [np.array(b, dtype=np.float64, copy=True) for b in boundary]
    A, rhs = assemble(w, prev_fields, boundary, 1, nx - 1, 1, ny - 1, Dt)
    lu = spla.splu(A)
    for f in range(len(out)):
        out[f][1:ny - 1, 1:nx - 1] = lu.solve(rhs[f]).reshape(ny - 2, nx - 2)
    return out


def dense_matrix(w, i0, i1, j0, j1, Dt):
    """The block's matrix as a dense array (for small brute-force checks)."""
    zeros = np.zeros_like(np.asarray(w, dtype=np.float64))
    A, _ = assemble(np.asarray(w, dtype=np.float64), [zeros], [zeros], i0, i1, j0, j1, Dt)
    return A.toarray()


def nonconservative_step(w, prev, boundary, Dt):
    """Implicit Euler of Eq. (3) written directly, -(1/w) grad w . grad xi + lap xi,
    with central differences for every derivative (including grad w), whole
    square, outer boundary Dirichlet. Used only to check reading R14: both
    discretisations approximate the same PDE and must agree to O(h^2)."""
    w = np.asarray(w, dtype=np.float64)
    ny, nx = w.shape
    hx = 1.0 / (nx - 1)
    hy = 1.0 / (ny - 1)
    mx, my = nx - 2, ny - 2
    m = mx * my
    rows, cols, vals = [], [], []
    rhs = np.zeros(m)

    def idx(i, j):
        return (j - 1) * mx + (i - 1)

    for j in range(1, ny - 1):
        for i in range(1, nx - 1):
            r = idx(i, j)
            bx = -(w[j, i + 1] - w[j, i - 1]) / (2 * hx) / w[j, i]
            by = -(w[j + 1, i] - w[j - 1, i]) / (2 * hy) / w[j, i]
            diag = 1.0 / Dt + 2.0 / hx ** 2 + 2.0 / hy ** 2
            rhs[r] += prev[j, i] / Dt
            for (di, dj, c) in ((-1, 0, 1 / hx ** 2 - bx / (2 * hx)), (1, 0, 1 / hx ** 2 + bx / (2 * hx)),
                                (0, -1, 1 / hy ** 2 - by / (2 * hy)), (0, 1, 1 / hy ** 2 + by / (2 * hy))):
                ii, jj = i + di, j + dj
                if 1 <= ii < nx - 1 and 1 <= jj < ny - 1:
                    rows.append(r)
                    cols.append(idx(ii, jj))
                    vals.append(-c)
                else:
                    rhs[r] += c * boundary[jj, ii]
            rows.append(r)
            cols.append(r)
            vals.append(diag)
    A = sp.csc_matrix((vals, (rows, cols)), shape=(m, m))
    out = np.array(boundary, dtype=np.float64, copy=True)
    out[1:ny - 1, 1:nx - 1] = spla.spsolve(A, rhs).reshape(my, mx)
    return out
