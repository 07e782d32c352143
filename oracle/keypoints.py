"""Key-point placement and interface fill of Sec. 4 (test infrastructure).

TEST INFRASTRUCTURE ONLY: used by the test suite; the product library never
imports it.

Sec. 4 computes the stochastic solution only at a few interface points, near
the maxima and minima of rho_x and rho_xx along the horizontal interfaces and
of rho_y and rho_yy along the vertical ones (rho = 1 / w, Sec. 5), and Sec. 5
recovers the other interface points by piecewise cubic Hermite interpolation.
Readings taken here (the paper gives no formulas):

  lines      vertical interface lines i = I_a, horizontal lines j = J_b, at
             I_a = floor(a (nx - 1) / sub_x + 1/2); a line's positions are its
             interior nodes t = 1 .. n - 2 (t = 0 and n - 1 lie on the boundary);
  profiles   along a line, the undivided differences of rho at t = 1 .. n - 2:
             D1(t) = rho(t + 1) - rho(t - 1)        (proportional to rho_s)
             D2(t) = (rho(t + 1) - rho(t)) - (rho(t) - rho(t - 1))  (to rho_ss)
             with rho = 1 / w in double precision;
  key points a position t in 2 .. n - 3 where D1 or D2 has a local extremum
             (p(t) > p(t - 1) and p(t) >= p(t + 1), or p(t) < p(t - 1) and
             p(t) <= p(t + 1)) of size |p(t)| >= max_t |p| / 100 -- the grid
             node nearest the extremum; smaller extrema (rounding noise where
             rho is flat) do not count -- every crossing of a vertical and
             a horizontal line, and, with spacing g > 0, every position t
             with t mod g = 0 (the mesh also moves where rho is flat along a
             line, and a fill through the extrema alone misses that);
  fill       along every line, the PCHIP interpolant (Fritsch and Carlson's
             monotone cubic Hermite scheme with the derivatives of Fritsch and
             Butland, as scipy.interpolate.PchipInterpolator implements it)
             through the two boundary values (the face data at t = 0, n - 1)
             and the key points' estimates, evaluated at the other positions.

The node list is the interface list of the estimator: vertical lines first,
bottom to top, then horizontal lines left to right without the crossings.
"""
from __future__ import annotations

import math

import numpy as np


def line_indices(n: int, parts: int):
    return [int(math.floor(k * (n - 1) / parts + 0.5)) for k in range(1, parts)]


def node_list(nx: int, ny: int, sub_x: int, sub_y: int):
    """(i, j) of the interface nodes in the estimator's order."""
    vi, hj = line_indices(nx, sub_x), line_indices(ny, sub_y)
    nodes = [(I, j) for I in vi for j in range(1, ny - 1)]
    vset = set(vi)
    nodes += [(i, J) for J in hj for i in range(1, nx - 1) if i not in vset]
    return nodes


def lines(nx: int, ny: int, sub_x: int, sub_y: int):
    """Each line as (orientation 'v'/'h', fixed index, [(i, j) for t = 0 .. n - 1])."""
    out = [("v", I, [(I, t) for t in range(ny)]) for I in line_indices(nx, sub_x)]
    out += [("h", J, [(t, J) for t in range(nx)]) for J in line_indices(ny, sub_y)]
    return out


def _extrema(p):
    """Positions (indices into p) of local extrema of at least a hundredth of the
    largest |p|, interior positions only."""
    big = max(abs(v) for v in p) if len(p) else 0.0
    out = []
    for k in range(1, len(p) - 1):
        if abs(p[k]) * 100.0 < big or big == 0.0:
            continue
        if (p[k] > p[k - 1] and p[k] >= p[k + 1]) or (p[k] < p[k - 1] and p[k] <= p[k + 1]):
            out.append(k)
    return out


def key_mask(w, sub_x: int, sub_y: int, spacing: int = 0):
    """Boolean mask over the interface node list: True at the key points."""
    w = np.asarray(w, dtype=np.float64)
    ny, nx = w.shape
    rho = 1.0 / w
    nodes = node_list(nx, ny, sub_x, sub_y)
    index = {nd: k for k, nd in enumerate(nodes)}
    mask = np.zeros(len(nodes), dtype=bool)
    vi, hj = set(line_indices(nx, sub_x)), set(line_indices(ny, sub_y))
    for orient, fixed, pts in lines(nx, ny, sub_x, sub_y):
        r = np.array([rho[j, i] for (i, j) in pts])
        n = len(pts)
        # profiles at t = 1 .. n - 2 (array position t - 1)
        d1 = [r[t + 1] - r[t - 1] for t in range(1, n - 1)]
        d2 = [(r[t + 1] - r[t]) - (r[t] - r[t - 1]) for t in range(1, n - 1)]
        for prof in (d1, d2):
            for k in _extrema(prof):
                mask[index[pts[k + 1]]] = True
        if spacing > 0:
            for t in range(1, n - 1):
                if t % spacing == 0:
                    mask[index[pts[t]]] = True
        for (i, j) in pts[1:-1]:
            if i in vi and j in hj:
                mask[index[(i, j)]] = True
    return mask


def pchip_fill(values_xi, values_eta, mask, faces, nx: int, ny: int, sub_x: int, sub_y: int):
    """Interface values with the non-key nodes filled by PCHIP along their lines.

    values_*: estimates over the node list (only the key entries are used);
    faces: the face data (layout of the estimator) giving the line ends."""
    from scipy.interpolate import PchipInterpolator
    from . import split_faces
    F = split_faces(np.asarray(faces, dtype=np.float64), nx, ny)
    nodes = node_list(nx, ny, sub_x, sub_y)
    index = {nd: k for k, nd in enumerate(nodes)}
    out = [np.array(values_xi, dtype=np.float64, copy=True), np.array(values_eta, dtype=np.float64, copy=True)]
    vi, hj = set(line_indices(nx, sub_x)), set(line_indices(ny, sub_y))
    for orient, fixed, pts in lines(nx, ny, sub_x, sub_y):
        n = len(pts)
        for f, vals in enumerate((values_xi, values_eta)):
            if orient == "v":
                ends = (F[(f, 2)][fixed], F[(f, 3)][fixed])     # bottom, top faces at column fixed
            else:
                ends = (F[(f, 0)][fixed], F[(f, 1)][fixed])     # left, right faces at row fixed
            xs, ys = [0.0], [ends[0]]
            for t in range(1, n - 1):
                k = index[pts[t]]
                if mask[k]:
                    xs.append(float(t))
                    ys.append(vals[k])
            xs.append(float(n - 1))
            ys.append(ends[1])
            P = PchipInterpolator(np.array(xs), np.array(ys))
            for t in range(1, n - 1):
                i, j = pts[t]
                if orient == "h" and i in vi:
                    continue                     # a crossing: owned by its vertical line (always key)
                k = index[pts[t]]
                if not mask[k]:
                    out[f][k] = float(P(float(t)))
    return out
