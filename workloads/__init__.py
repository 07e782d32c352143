"""Seeded synthetic inputs for the interface Monte Carlo workloads.

This module only builds inputs: grids, mesh-density fields w sampled from the
analytic formulas of the workloads, initial fields and interface node lists.
It holds none of the method's arithmetic (no drift, no face data, no
estimator), so both the CUDA path's callers and the CPU oracle can draw their
inputs from it.

Workloads (all on the unit square, xi0 = x and eta0 = y unless stated):

  heat65      w = 1 on 65 x 65; xi0 = sin(pi x) sin(pi y), eta0 = sin(pi x) sin(2 pi y);
              zero boundary data; 33 nodes x = 1/2, y = j/32; 1000 paths;
              dt = 1e-3, Delta t = 0.05; seed 0.
  front257    w = 1 + 10 exp(-(x - 0.3 - 0.4 t)^2 / 0.05^2) on 257 x 257 (FP32),
              2 x 2 subdomains, 509 interface nodes, 1e4 paths, dt = 1e-4,
              Delta t = 1e-2, 50 mesh steps.
  batch64     64 instances, Gaussian-bump w, grids 65..513, 33..1023 nodes,
              1e3..1e5 paths (log-uniform), dt = 1e-4, Delta t = 1e-2.
  ring2049    w = 1 + 50 exp(-(r - 0.25 - 0.1 sin 2 pi t)^2 / 0.02^2) on 2049 x 2049,
              8 x 8 subdomains, 28,609 interface nodes, 2e4 paths, dt = 1e-5,
              Delta t = 1e-3, 20 mesh steps.
  ring41      the paper's experiment (Sec. 5): w = 1 / rho with
              rho = 1 + 10 exp(-50 |(x - 1/2 - cos(2 pi t)/4)^2 + (y - 1/2 - sin(2 pi t)/4)^2 - 1/100|),
              41 x 41, 2 x 2 subdomains, Delta t = 1e-3, 20 sub-steps, 1e4 paths.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def grid(nx: int, ny: int | None = None):
    """Node coordinates X[j, i] = i / (nx - 1), Y[j, i] = j / (ny - 1)."""
    ny = nx if ny is None else ny
    x = np.arange(nx, dtype=np.float64) / (nx - 1)
    y = np.arange(ny, dtype=np.float64) / (ny - 1)
    X, Y = np.meshgrid(x, y)
    return X, Y


def identity_fields(nx: int, ny: int | None = None):
    """xi0 = x, eta0 = y: the uniform initial mesh (Sec. 3)."""
    X, Y = grid(nx, ny)
    return X.copy(), Y.copy()


# ---------------------------------------------------------------- w fields

def w_const(nx: int, ny: int | None = None, value: float = 1.0):
    ny = nx if ny is None else ny
    return np.full((ny, nx), value, dtype=np.float32)


def w_front(n: int, t: float):
    """Moving front, sampled at time t, stored as FP32."""
    X, Y = grid(n)
    return (1.0 + 10.0 * np.exp(-((X - 0.3 - 0.4 * t) ** 2) / 0.05 ** 2)).astype(np.float32)


def w_ring(n: int, t: float):
    """Ring front of radius 0.25 + 0.1 sin(2 pi t), sampled at time t, FP32."""
    X, Y = grid(n)
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2)
    return (1.0 + 50.0 * np.exp(-((r - 0.25 - 0.1 * math.sin(2 * math.pi * t)) ** 2) / 0.02 ** 2)).astype(
        np.float32)


def w_bump(n: int, cx: float, cy: float, width: float, alpha: float):
    """Gaussian bump 1 + alpha exp(-|x - c|^2 / width^2), FP32."""
    X, Y = grid(n)
    return (1.0 + alpha * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / width ** 2)).astype(np.float32)


def w_paper_ring(n: int, t: float):
    """The paper's Sec. 5 weight w = 1 / rho (alpha = 10, beta = -50), FP32."""
    X, Y = grid(n)
    q = (X - 0.5 - 0.25 * math.cos(2 * math.pi * t)) ** 2 + (Y - 0.5 - 0.25 * math.sin(2 * math.pi * t)) ** 2
    rho = 1.0 + 10.0 * np.exp(-50.0 * np.abs(q - 0.01))
    return (1.0 / rho).astype(np.float32)


def w_smooth_random(n: int, seed: int, modes: int = 3, amp: float = 0.4):
    """A smooth positive random field (a few low Fourier modes), for parity tests."""
    rng = np.random.default_rng(seed)
    X, Y = grid(n)
    w = np.ones_like(X)
    for _ in range(modes):
        kx, ky = rng.integers(1, 4, size=2)
        ph = rng.uniform(0, 2 * math.pi, size=2)
        w += amp / modes * rng.uniform(-1, 1) * np.cos(math.pi * kx * X + ph[0]) * np.cos(math.pi * ky * Y + ph[1])
    return w.astype(np.float32)


# ------------------------------------------------------------ node sets

def interface_lines(n_nodes: int, n_sub: int):
    """Grid indices of the interface lines splitting n_nodes nodes into n_sub parts."""
    # nearest index, halves rounded up
    return [int(math.floor(k * (n_nodes - 1) / n_sub + 0.5)) for k in range(1, n_sub)]


def interface_nodes(nx: int, ny: int, sub_x: int, sub_y: int):
    """Interior nodes of the interface lines, each once (reading R15).

    Order: the vertical lines i = I_1 < I_2 < ... first, each bottom to top
    (j = 1 .. ny-2); then the horizontal lines j = J_1 < ..., left to right
    (i = 1 .. nx-2), skipping nodes that lie on a vertical line.
    Returns (i, j) integer arrays.
    """
    vi = interface_lines(nx, sub_x)
    hj = interface_lines(ny, sub_y)
    ii, jj = [], []
    for I in vi:
        for j in range(1, ny - 1):
            ii.append(I)
            jj.append(j)
    vset = set(vi)
    for J in hj:
        for i in range(1, nx - 1):
            if i in vset:
                continue
            ii.append(i)
            jj.append(J)
    return np.array(ii, dtype=np.int64), np.array(jj, dtype=np.int64)


def interface_node_coords(nx: int, ny: int, sub_x: int, sub_y: int):
    i, j = interface_nodes(nx, ny, sub_x, sub_y)
    return i / (nx - 1), j / (ny - 1)


def heat65_nodes():
    """33 nodes on x = 1/2 at y = j/32, j = 0..32 (the two ends lie on the boundary)."""
    y = np.arange(33, dtype=np.float64) / 32.0
    return np.full(33, 0.5), y


# ------------------------------------------------------------ workloads

@dataclass
class Workload:
    name: str
    n: int
    sub: int
    dt: float
    Dt: float
    paths: int
    steps: int
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def K(self):
        return int(round(self.Dt / self.dt))


HEAT65 = Workload("heat65", n=65, sub=2, dt=1e-3, Dt=0.05, paths=1000, steps=1)
FRONT257 = Workload("front257", n=257, sub=2, dt=1e-4, Dt=1e-2, paths=10000, steps=50)
RING2049 = Workload("ring2049", n=2049, sub=8, dt=1e-5, Dt=1e-3, paths=20000, steps=20)
RING41 = Workload("ring41", n=41, sub=2, dt=5e-5, Dt=1e-3, paths=10000, steps=750)


def heat65_fields():
    X, Y = grid(65)
    xi0 = np.sin(np.pi * X) * np.sin(np.pi * Y)
    eta0 = np.sin(np.pi * X) * np.sin(2 * np.pi * Y)
    return xi0, eta0


def heat_exact(x, y, t):
    """Closed forms of the w = 1 heat problem from heat65_fields: separable Fourier modes."""
    xi = math.exp(-2 * math.pi ** 2 * t) * np.sin(np.pi * x) * np.sin(np.pi * y)
    eta = math.exp(-5 * math.pi ** 2 * t) * np.sin(np.pi * x) * np.sin(2 * np.pi * y)
    return xi, eta


@dataclass
class Instance:
    n: int
    cx: float
    cy: float
    width: float
    alpha: float
    nodes_i: np.ndarray
    nodes_j: np.ndarray
    paths: np.ndarray


def batch64_instances(seed: int = 0, count: int = 64):
    """64 independent Gaussian-bump instances (reading R18).

    Per instance: n in {65, 129, 257, 513}; centre ~ U[0.2, 0.8]^2; width ~
    U[0.05, 0.15]; alpha ~ U[1, 50]; node count log-uniform in [33, 1023],
    taken evenly from the instance's 2 x 2 interface node list; paths per node
    log-uniform in [1e3, 1e5]. Instance i draws from seed + i.
    """
    out = []
    for k in range(count):
        rng = np.random.default_rng(seed + k)
        n = int(rng.choice([65, 129, 257, 513]))
        cx, cy = rng.uniform(0.2, 0.8, size=2)
        width = rng.uniform(0.05, 0.15)
        alpha = rng.uniform(1.0, 50.0)
        ii, jj = interface_nodes(n, n, 2, 2)
        want = int(round(math.exp(rng.uniform(math.log(33), math.log(1023)))))
        want = max(1, min(want, ii.size))
        pick = np.unique(np.linspace(0, ii.size - 1, want).round().astype(np.int64))
        paths = np.exp(rng.uniform(math.log(1e3), math.log(1e5), size=pick.size)).round().astype(np.int64)
        out.append(Instance(n, float(cx), float(cy), float(width), float(alpha), ii[pick], jj[pick], paths))
    return out
