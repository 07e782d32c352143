"""FP64 CPU oracle of the interface Monte Carlo method (test infrastructure).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers. The product library never imports,
loads or runs anything in this directory, and this directory imports nothing
from the product package.

Layout:
  sdd_oracle.c  plain C, double precision: Philox4x32-10 + Box--Muller, the
                finite-difference drift, bilinear interpolation, the 1D
                Winslow face data and the path-by-path estimator of Eq. (7b).
  solver.py     the implicit finite-difference subdomain solve (Sec. 4), by
                sparse LU as in the paper.
  mlp.py        double-precision forward/backward of the control-variate
                network.

Every function here restates the paper's definition or algorithm; no part of
it is blocked, fused or reordered for speed.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile sdd_oracle.c into oracle/_build/liboracle.so (gcc, -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("bx", ctypes.c_void_p), ("by", ctypes.c_void_p),
                ("xi0", ctypes.c_void_p), ("eta0", ctypes.c_void_p),
                ("faces", ctypes.c_void_p), ("cv", ctypes.c_void_p), ("cv_slices", ctypes.c_int),
                ("cv_cell", ctypes.c_int)]


class _Params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("K", ctypes.c_int32), ("exit_mode", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("step_index", ctypes.c_uint32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp = ctypes.c_void_p
            lib.orc_philox4x32_10.argtypes = [vp, vp, vp]
            lib.orc_box_muller.argtypes = [ctypes.c_uint32, ctypes.c_uint32, vp, vp]
            lib.orc_drift_field.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp]
            lib.orc_bilinear.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.c_double, ctypes.c_double]
            lib.orc_bilinear.restype = ctypes.c_double
            lib.orc_winslow_faces.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp]
            lib.orc_faces_len.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.orc_faces_len.restype = ctypes.c_int64
            lib.orc_face_value.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double]
            lib.orc_face_value.restype = ctypes.c_double
            lib.orc_mc_nodes.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(_Params), ctypes.c_int64,
                                         vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            lib.orc_mc_nodes.restype = ctypes.c_int
            lib.orc_draw.argtypes = [ctypes.c_uint64, ctypes.c_int64, vp, vp, vp]
            lib.orc_path_margins.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(_Params), ctypes.c_int64,
                                             vp, vp, vp, vp, vp, vp]
            lib.orc_path_margins.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


# --------------------------------------------------------------------------
# Variates
# --------------------------------------------------------------------------

def philox4x32_10(ctr, key):
    """One Philox4x32-10 block (SC'11) for a 4-word counter and 2-word key."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib.orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def box_muller(a: int, b: int):
    """Box--Muller pair from two words: (R cos 2 pi U2, R sin 2 pi U2)."""
    lib = _load()
    z0 = np.zeros(1)
    z1 = np.zeros(1)
    lib.orc_box_muller(ctypes.c_uint32(a), ctypes.c_uint32(b), _p(z0), _p(z1))
    return float(z0[0]), float(z1[0])


def draw(seed: int, counters):
    """Philox words and normals for counters (path, node, draw, step), shape (n, 4).

    Returns (words (n,4) uint32, normals (n,4) float64): normals[:, 0:2] from
    words 0,1 and normals[:, 2:4] from words 2,3.
    """
    lib = _load()
    c = np.ascontiguousarray(counters, dtype=np.uint32).reshape(-1, 4)
    n = c.shape[0]
    words = np.zeros((n, 4), np.uint32)
    normals = np.zeros((n, 4), np.float64)
    lib.orc_draw(ctypes.c_uint64(seed), ctypes.c_int64(n), _p(c), _p(words), _p(normals))
    return words, normals


# --------------------------------------------------------------------------
# Fields
# --------------------------------------------------------------------------

def drift_field(w):
    """b = -grad w / w at the nodes by finite differences (Eq. 6, Sec. 4)."""
    lib = _load()
    w = np.ascontiguousarray(w, dtype=np.float64)
    ny, nx = w.shape
    bx = np.zeros_like(w)
    by = np.zeros_like(w)
    lib.orc_drift_field(nx, ny, _p(w), _p(bx), _p(by))
    return bx, by


def bilinear(f, x: float, y: float) -> float:
    """Bilinear interpolation of node values f[j, i] at (x, y) (Sec. 4)."""
    lib = _load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    ny, nx = f.shape
    return float(lib.orc_bilinear(nx, ny, _p(f), x, y))


def faces_len(nx: int, ny: int) -> int:
    return 2 * (2 * ny + 2 * nx)


def winslow_faces(w):
    """Face data of Sec. 3: 0/1 on two faces, the 1D Winslow solution on the others."""
    lib = _load()
    w = np.ascontiguousarray(w, dtype=np.float64)
    ny, nx = w.shape
    faces = np.zeros(faces_len(nx, ny))
    lib.orc_winslow_faces(nx, ny, _p(w), _p(faces))
    return faces


def face_value(faces, nx: int, ny: int, field: int, face: int, s: float) -> float:
    lib = _load()
    faces = np.ascontiguousarray(faces, dtype=np.float64)
    return float(lib.orc_face_value(nx, ny, _p(faces), field, face, s))


def split_faces(faces, nx: int, ny: int):
    """Name the 8 face segments: {(field, face): array}."""
    out = {}
    off = 0
    for field in (0, 1):
        for face, n in ((0, ny), (1, ny), (2, nx), (3, nx)):
            out[(field, face)] = faces[off:off + n]
            off += n
    return out


# --------------------------------------------------------------------------
# The estimator
# --------------------------------------------------------------------------

@dataclass
class Problem:
    """One mesh step's data: w at t_{n-1} (as the GPU receives it), xi, eta at t_{n-1}, faces."""
    w: np.ndarray           # (ny, nx); widened to FP64
    xi0: np.ndarray         # (ny, nx) FP64
    eta0: np.ndarray        # (ny, nx) FP64
    faces: np.ndarray | None = None   # None: Winslow 1D data from w

    def __post_init__(self):
        self.w = np.ascontiguousarray(self.w, dtype=np.float64)
        self.xi0 = np.ascontiguousarray(self.xi0, dtype=np.float64)
        self.eta0 = np.ascontiguousarray(self.eta0, dtype=np.float64)
        if self.faces is None:
            self.faces = winslow_faces(self.w)
        self.faces = np.ascontiguousarray(self.faces, dtype=np.float64)
        self.bx, self.by = drift_field(self.w)

    @property
    def ny(self):
        return self.w.shape[0]

    @property
    def nx(self):
        return self.w.shape[1]


def sub_steps(dt: float, Dt: float) -> int:
    """K = Delta t / dt, which must be an integer (Sec. 4 sub-time steps)."""
    K = int(round(Dt / dt))
    if K < 1 or abs(K * dt - Dt) > 1e-9 * Dt:
        raise ValueError("Delta t must be an integer multiple of dt")
    return K


def interface_mc(problem: Problem, xs, ys, n_paths, *, dt: float, Dt: float, seed: int = 0,
                 exit_mode: int = 0, step_index: int = 0, node_ids=None,
                 record: bool = False, threads: int | None = None, cv_table=None):
    """Estimate xi, eta at the given nodes over one mesh step (Eq. 7b, Sec. 4).

    exit_mode: 0 fixed sub-steps with the plain exit test, 1 fixed sub-steps
    with the plain and the Brownian-bridge tests, 2 exponential time-stepping
    (sub-step lengths exponential with mean dt, both tests over each).

    Returns a dict with mean_xi, mean_eta, se_xi, se_eta, n_exit, path_steps
    (one entry per node) and, with record=True, per-path arrays steps, code,
    score_xi, score_eta, x_end, y_end laid out node after node.
    node_ids: each node's word in the Philox counter (default 0..count-1).
    threads: worker threads over nodes (ctypes releases the GIL), default all cores.
    cv_table: optional control-variate model gradients, shape (S, ny, nx, 4):
    slice q serves the sub-steps j with floor(j S / K) = q; components are
    d/dx, d/dy of the xi model and of the eta model at the nodes, interpolated
    bilinearly; or shape (1, ny - 1, nx - 1, 4): one value per cell, the model
    at a point being the value of its cell.
    """
    lib = _load()
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    ys = np.ascontiguousarray(ys, dtype=np.float64)
    count = xs.shape[0]
    n_paths = np.ascontiguousarray(np.broadcast_to(np.asarray(n_paths, dtype=np.int64), (count,)))
    if node_ids is None:
        node_ids = np.arange(count, dtype=np.uint32)
    node_ids = np.ascontiguousarray(node_ids, dtype=np.uint32)
    K = sub_steps(dt, Dt)
    cv = None
    if cv_table is not None:
        if exit_mode == 2:
            raise ValueError("the control variate needs fixed sub-steps (exit_mode 0 or 1)")
        cv = np.ascontiguousarray(cv_table, dtype=np.float64)
        cell = cv.shape[1:] == (problem.ny - 1, problem.nx - 1, 4)
        assert cv.ndim == 4 and (cv.shape[1:] == (problem.ny, problem.nx, 4) or (cell and cv.shape[0] == 1))
    P = _Problem(problem.nx, problem.ny, problem.bx.ctypes.data, problem.by.ctypes.data,
                 problem.xi0.ctypes.data, problem.eta0.ctypes.data, problem.faces.ctypes.data,
                 cv.ctypes.data if cv is not None else None, cv.shape[0] if cv is not None else 0,
                 1 if cv is not None and cell else 0)
    Q = _Params(dt, K, exit_mode, seed, step_index)
    stats = np.zeros((count, 6))
    total = int(n_paths.sum())
    recs = None
    if record:
        recs = dict(steps=np.zeros(total, np.int32), code=np.zeros(total, np.int32),
                    score_xi=np.zeros(total), score_eta=np.zeros(total),
                    x_end=np.zeros(total), y_end=np.zeros(total))
    offs = np.concatenate([[0], np.cumsum(n_paths)])
    threads = threads or (os.cpu_count() or 1)
    nchunk = max(1, min(count, threads * 4))
    bounds = np.linspace(0, count, nchunk + 1).astype(np.int64)

    def run(c):
        a, b = int(bounds[c]), int(bounds[c + 1])
        if a == b:
            return 0
        def at(arr, itemsize, off):
            return ctypes.c_void_p(arr.ctypes.data + itemsize * off) if arr is not None else ctypes.c_void_p(0)
        r0 = int(offs[a])
        rp = [None] * 6
        if recs is not None:
            rp = [at(recs["steps"], 4, r0), at(recs["code"], 4, r0), at(recs["score_xi"], 8, r0),
                  at(recs["score_eta"], 8, r0), at(recs["x_end"], 8, r0), at(recs["y_end"], 8, r0)]
        else:
            rp = [ctypes.c_void_p(0)] * 6
        return lib.orc_mc_nodes(ctypes.byref(P), ctypes.byref(Q), ctypes.c_int64(b - a),
                                at(xs, 8, a), at(ys, 8, a), at(n_paths, 8, a), at(node_ids, 4, a),
                                at(stats, 48, a), *rp)

    if threads == 1 or nchunk == 1:
        rcs = [run(c) for c in range(nchunk)]
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            rcs = list(ex.map(run, range(nchunk)))
    if any(rc != 0 for rc in rcs):
        raise MemoryError("oracle ran out of memory")
    out = dict(mean_xi=stats[:, 0].copy(), mean_eta=stats[:, 1].copy(), se_xi=stats[:, 2].copy(),
               se_eta=stats[:, 3].copy(), n_exit=stats[:, 4].astype(np.int64),
               path_steps=stats[:, 5].astype(np.int64))
    if recs is not None:
        out.update(recs)
    return out


def path_margins(problem: Problem, xs, ys, node_ids, paths, upto, *, dt: float, Dt: float, seed: int = 0,
                 exit_mode: int = 0, step_index: int = 0):
    """For single paths (node coordinates xs, ys, Philox node words node_ids,
    path numbers paths): the smallest distance min(|x|, |1-x|, |y|, |1-y|) of
    the path's points X_1 .. X_s to the boundary lines, s = min(its sub-steps,
    upto). Test support: where another implementation's exit decision differs
    from the oracle's, the oracle's path must have come close to the boundary
    by then. Fixed sub-steps only (exit_mode 0 or 1)."""
    lib = _load()
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    ys = np.ascontiguousarray(ys, dtype=np.float64)
    node_ids = np.ascontiguousarray(node_ids, dtype=np.uint32)
    paths = np.ascontiguousarray(paths, dtype=np.uint32)
    upto = np.ascontiguousarray(upto, dtype=np.int32)
    count = xs.shape[0]
    assert ys.shape[0] == count and node_ids.shape[0] == count and paths.shape[0] == count and upto.shape[0] == count
    if exit_mode == 2:
        raise ValueError("margins are defined for fixed sub-steps (exit_mode 0 or 1)")
    P = _Problem(problem.nx, problem.ny, problem.bx.ctypes.data, problem.by.ctypes.data,
                 problem.xi0.ctypes.data, problem.eta0.ctypes.data, problem.faces.ctypes.data, None, 0, 0)
    Q = _Params(dt, sub_steps(dt, Dt), exit_mode, seed, step_index)
    out = np.full(count, np.inf)
    if count:
        rc = lib.orc_path_margins(ctypes.byref(P), ctypes.byref(Q), ctypes.c_int64(count), _p(xs), _p(ys),
                                  _p(node_ids), _p(paths), _p(upto), _p(out))
        assert rc == 0
    return out


# --------------------------------------------------------------------------
# One mesh step of the decomposition method
# --------------------------------------------------------------------------

def boundary_grid(faces, nx: int, ny: int, field: int, inner):
    """A grid holding `inner` inside and the face data on the boundary ring
    (left, right, bottom, top: the first that holds wins at the corners)."""
    seg = split_faces(faces, nx, ny)
    g = np.array(inner, dtype=np.float64, copy=True)
    g[-1, :] = seg[(field, 3)]
    g[0, :] = seg[(field, 2)]
    g[:, -1] = seg[(field, 1)]
    g[:, 0] = seg[(field, 0)]
    return g


def dd_step(w, xi, eta, *, sub_x: int, sub_y: int, dt: float, Dt: float, n_paths: int, seed: int,
            step_index: int, nodes_ij, exit_mode: int = 0, faces=None, threads=None, node_word0: int = 0,
            cv_table=None, keypoints: bool = False, key_spacing: int = 0):
    """One mesh step t_{n-1} -> t_n of the method (Sec. 4): the interface
    estimate at the nodes nodes_ij = (i, j) (their position is their node index
    in the random stream), then the implicit subdomain solves by LU with those
    values and the face data as Dirichlet data. node_word0 offsets the node
    word of the random stream (instances evaluated together number their nodes
    in sequence); cv_table, if given, is the control variate of interface_mc. keypoints: estimate only at the key points of Sec. 4 and fill
    the rest of each interface line by PCHIP (oracle.keypoints; nodes_ij must
    then be the whole interface list; key_spacing adds every key_spacing-th
    position of each line). Returns ([xi_n, eta_n], stats)."""
    from . import solver
    P = Problem(w, xi, eta, faces)
    ii, jj = (np.asarray(a) for a in nodes_ij)
    xs = ii / (P.nx - 1)
    ys = jj / (P.ny - 1)
    ids = np.arange(xs.size, dtype=np.uint32) + np.uint32(node_word0)
    if keypoints:
        from . import keypoints as kp
        mask = kp.key_mask(P.w, sub_x, sub_y, key_spacing)
        assert mask.size == xs.size
        rk = interface_mc(P, xs[mask], ys[mask], n_paths, dt=dt, Dt=Dt, seed=seed, exit_mode=exit_mode,
                          step_index=step_index, threads=threads, node_ids=ids[mask], cv_table=cv_table)
        r = {k: np.zeros(xs.size, dtype=v.dtype) for k, v in rk.items() if np.ndim(v) == 1 and len(v) == mask.sum()}
        for k in r:
            r[k][mask] = rk[k]
        r["mean_xi"], r["mean_eta"] = kp.pchip_fill(r["mean_xi"], r["mean_eta"], mask, P.faces, P.nx, P.ny, sub_x,
                                                    sub_y)
        r["key"] = mask
    else:
        r = interface_mc(P, xs, ys, n_paths, dt=dt, Dt=Dt, seed=seed, exit_mode=exit_mode, step_index=step_index,
                         threads=threads, node_ids=ids, cv_table=cv_table)
    bx = boundary_grid(P.faces, P.nx, P.ny, 0, P.xi0)
    be = boundary_grid(P.faces, P.nx, P.ny, 1, P.eta0)
    bx[jj, ii] = r["mean_xi"]
    be[jj, ii] = r["mean_eta"]
    new = solver.subdomain_solve(P.w, [P.xi0, P.eta0], [bx, be], sub_x, sub_y, Dt)
    return new, r
