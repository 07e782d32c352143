"""Python binding of libsdd (include/sdd.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module only
turns torch tensors into device pointers, allocates outputs with torch and
checks status codes. There is no CPU fallback: if the library is missing the
first call raises.

    import torch, paper_1402_0266_gb300 as sdd
    ctx = sdd.sdd_init(nx=257, ny=257, sub_x=2, sub_y=2, w=w_dev)   # w: cuda float32 (ny, nx)
    out = sdd.sdd_interface_mc(ctx, x, y, n_paths, dt=1e-4, Dt=1e-2, seed=0)
    sdd.sdd_step(ctx, dt=1e-4, Dt=1e-2, seed=0, paths_per_node=10000)
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsdd.so")

SDD_OK, SDD_EINVAL, SDD_ENOMEM, SDD_ECUDA, SDD_ENOCONV, SDD_ETIMEOUT, SDD_EDEVICE = range(7)
STATUS_NAMES = {0: "SDD_OK", 1: "SDD_EINVAL", 2: "SDD_ENOMEM", 3: "SDD_ECUDA", 4: "SDD_ENOCONV",
                5: "SDD_ETIMEOUT", 6: "SDD_EDEVICE"}

# every entry point declared in include/sdd.h
EXPORTS = [
    "sdd_init", "sdd_set_w", "sdd_set_w_host", "sdd_set_fields", "sdd_set_boundary", "sdd_get_faces",
    "sdd_get_fields", "sdd_get_fields_host", "sdd_interface_mc", "sdd_interface_mc_record", "sdd_interface_nodes",
    "sdd_subdomain_solve", "sdd_step", "sdd_last_interface_stats", "sdd_last_step_info", "sdd_set_step_index",
    "sdd_get_step_index",
    "sdd_sync", "sdd_flush", "sdd_set_pipeline", "sdd_pipeline_in_use", "sdd_last_error", "sdd_destroy", "sdd_rng_draw", "sdd_interface_mc_static",
    "sdd_static_scratch_bytes", "sdd_batch_create", "sdd_batch_interface_mc", "sdd_batch_step",
    "sdd_batch_last_step_info", "sdd_batch_set_step_index", "sdd_batch_sync", "sdd_batch_last_error",
    "sdd_batch_destroy", "sdd_autotune", "sdd_batch_autotune", "sdd_cv_set_table", "sdd_cv_enable",
    "sdd_mlp_init", "sdd_cv_samples", "sdd_mlp_norm", "sdd_mlp_grad", "sdd_mlp_train", "sdd_cv_tabulate",
    "sdd_cv_train", "sdd_cv_get_model", "sdd_cv_losses", "sdd_cv_get_table", "sdd_cv_set_model",
    "sdd_cv_set_fields_order", "sdd_cv_fields_order", "sdd_cv_get_cells",
    "sdd_set_solver", "sdd_solver_in_use", "sdd_set_keypoints", "sdd_keypoint_mask", "sdd_keypoint_fill",
]

SDD_SOLVER_AUTO, SDD_SOLVER_JACOBI, SDD_SOLVER_MG, SDD_SOLVER_DIRECT = range(4)

SDD_CV_OFF, SDD_CV_TABLE, SDD_CV_MODEL, SDD_CV_FIELDS = range(4)

MLP_INPUTS, MLP_HIDDEN, MLP_PARAMS, MLP_STRIDE = 5, 64, 4609, 4616


class SddError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("sub_x", ctypes.c_int32), ("sub_y", ctypes.c_int32)]


class _Nodes(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("n_paths", ctypes.c_void_p), ("count", ctypes.c_int64)]


class _Stats(ctypes.Structure):
    _fields_ = [("mean_xi", ctypes.c_void_p), ("mean_eta", ctypes.c_void_p), ("se_xi", ctypes.c_void_p),
                ("se_eta", ctypes.c_void_p), ("n_exit", ctypes.c_void_p), ("path_steps", ctypes.c_void_p)]


class _Records(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_void_p), ("code", ctypes.c_void_p), ("score_xi", ctypes.c_void_p),
                ("score_eta", ctypes.c_void_p), ("x_end", ctypes.c_void_p), ("y_end", ctypes.c_void_p)]


class _McParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("Dt", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("step_index", ctypes.c_uint32), ("exit_mode", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("paths_per_task", ctypes.c_int32), ("node_word0", ctypes.c_uint32), ("zero_map", ctypes.c_int32)]


class _Fields(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("w", ctypes.c_void_p), ("xi", ctypes.c_void_p),
                ("eta", ctypes.c_void_p), ("faces", ctypes.c_void_p)]


class _StepInfo(ctypes.Structure):
    _fields_ = [("kernel_nodes", ctypes.c_int32), ("paths_ms", ctypes.c_float), ("estimate_ms", ctypes.c_float),
                ("solve_ms", ctypes.c_float), ("step_ms", ctypes.c_float)]


class _StepParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("Dt", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("paths_per_node", ctypes.c_int64), ("exit_mode", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("rtol", ctypes.c_double), ("tune", ctypes.c_int32), ("pad", ctypes.c_int32)]


class _Shape(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("paths_per_task", ctypes.c_int32), ("ms", ctypes.c_float),
                ("zero_map", ctypes.c_int32)]


class _SampleParams(ctypes.Structure):
    _fields_ = [("per_horizon", ctypes.c_int32), ("exit_mode", ctypes.c_int32), ("dt", ctypes.c_double),
                ("Dt", ctypes.c_double), ("seed", ctypes.c_uint64)]


class _TrainParams(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_double),
                ("max_steps", ctypes.c_int64)]


class _CvTrainParams(ctypes.Structure):
    _fields_ = [("samples", _SampleParams), ("train", _TrainParams), ("slices", ctypes.c_int32),
                ("warm_start", ctypes.c_int32), ("init_seed", ctypes.c_uint64)]


class _CvTrainInfo(ctypes.Structure):
    _fields_ = [("samples_ms", ctypes.c_float), ("train_ms", ctypes.c_float), ("tabulate_ms", ctypes.c_float),
                ("loss_xi", ctypes.c_float), ("loss_eta", ctypes.c_float), ("slices", ctypes.c_int32),
                ("rows", ctypes.c_int64), ("steps", ctypes.c_int64)]


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded libsdd.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libsdd.so not found at {LIB_PATH}: build it with "
                                   "`python -m paper_1402_0266_gb300.build` (no CPU fallback exists)")
            L = ctypes.CDLL(LIB_PATH)
            vp, i32, i64, u32, u64, dbl = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                           ctypes.c_uint64, ctypes.c_double)
            sig = {
                "sdd_init": [ctypes.POINTER(vp), ctypes.POINTER(_Grid), vp, vp, vp, vp],
                "sdd_set_w": [vp, vp],
                "sdd_set_w_host": [vp, vp],
                "sdd_set_fields": [vp, vp, vp],
                "sdd_set_boundary": [vp, vp],
                "sdd_get_faces": [vp, vp],
                "sdd_get_fields": [vp, vp, vp],
                "sdd_get_fields_host": [vp, vp, vp],
                "sdd_interface_mc": [vp, ctypes.POINTER(_Nodes), ctypes.POINTER(_McParams), ctypes.POINTER(_Stats)],
                "sdd_interface_mc_record": [vp, ctypes.POINTER(_Nodes), ctypes.POINTER(_McParams),
                                            ctypes.POINTER(_Stats), ctypes.POINTER(_Records)],
                "sdd_interface_nodes": [vp, vp, vp, ctypes.POINTER(i64)],
                "sdd_subdomain_solve": [vp, dbl, vp, vp, dbl, i32, vp, vp, ctypes.POINTER(i32)],
                "sdd_step": [vp, ctypes.POINTER(_StepParams)],
                "sdd_last_interface_stats": [vp, ctypes.POINTER(_Stats)],
                "sdd_last_step_info": [vp, ctypes.POINTER(_StepInfo)],
                "sdd_set_step_index": [vp, u32],
                "sdd_get_step_index": [vp],
                "sdd_sync": [vp],
                "sdd_flush": [vp],
                "sdd_set_pipeline": [vp, ctypes.c_int32],
                "sdd_last_error": [vp],
                "sdd_destroy": [vp],
                "sdd_rng_draw": [u64, vp, i64, vp, vp, vp],
                "sdd_interface_mc_static": [ctypes.POINTER(_Fields), ctypes.POINTER(_Nodes), ctypes.POINTER(_McParams),
                                            ctypes.POINTER(_Stats), vp, vp],
                "sdd_static_scratch_bytes": [],
                "sdd_batch_create": [ctypes.POINTER(vp), ctypes.POINTER(vp), i32, vp],
                "sdd_batch_interface_mc": [vp, ctypes.POINTER(_Nodes), ctypes.POINTER(_McParams),
                                           ctypes.POINTER(_Stats)],
                "sdd_batch_step": [vp, ctypes.POINTER(_StepParams)],
                "sdd_batch_last_step_info": [vp, ctypes.POINTER(_StepInfo)],
                "sdd_batch_set_step_index": [vp, u32],
                "sdd_batch_sync": [vp],
                "sdd_batch_last_error": [vp],
                "sdd_batch_destroy": [vp],
                "sdd_autotune": [vp, ctypes.POINTER(_Nodes), ctypes.POINTER(_McParams), ctypes.POINTER(_Shape)],
                "sdd_cv_set_table": [vp, vp, i32],
                "sdd_cv_enable": [vp, i32],
                "sdd_mlp_init": [vp, u64, vp],
                "sdd_cv_samples": [vp, ctypes.POINTER(_SampleParams), vp, vp],
                "sdd_mlp_norm": [vp, vp, i64, vp],
                "sdd_mlp_grad": [vp, vp, vp, vp, vp, i64, vp, vp],
                "sdd_mlp_train": [vp, vp, vp, vp, vp, i64, ctypes.POINTER(_TrainParams), vp],
                "sdd_cv_tabulate": [vp, vp, vp, i32, dbl, dbl],
                "sdd_cv_train": [vp, ctypes.POINTER(_CvTrainParams), ctypes.POINTER(_CvTrainInfo)],
                "sdd_cv_get_model": [vp, vp, vp],
                "sdd_cv_losses": [vp, vp, i64],
                "sdd_cv_get_table": [vp, vp],
                "sdd_cv_set_fields_order": [vp, i32],
                "sdd_cv_get_cells": [vp, vp],
                "sdd_cv_set_model": [vp, vp, vp, i32],
                "sdd_set_solver": [vp, i32],
                "sdd_set_keypoints": [vp, i32, i32],
                "sdd_keypoint_mask": [vp, vp],
                "sdd_keypoint_fill": [vp, vp, vp, vp],
                "sdd_solver_in_use": [vp],
                "sdd_pipeline_in_use": [vp],
                "sdd_batch_autotune": [vp, ctypes.POINTER(_Nodes), ctypes.POINTER(_McParams), ctypes.POINTER(_Shape)],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            L.sdd_get_step_index.restype = ctypes.c_uint32
            L.sdd_cv_fields_order.argtypes = [vp]
            L.sdd_cv_fields_order.restype = ctypes.c_int32
            L.sdd_static_scratch_bytes.restype = ctypes.c_int64
            L.sdd_batch_last_error.restype = ctypes.c_char_p
            L.sdd_batch_destroy.restype = None
            L.sdd_last_error.restype = ctypes.c_char_p
            L.sdd_destroy.restype = None
            _lib = L
    return _lib


def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(0) if t is None else ctypes.c_void_p(t.data_ptr())


def _check_dev(t, dtype, shape, name):
    torch = _torch()
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name}: expected a contiguous cuda {dtype} tensor")
    if shape is not None and tuple(t.shape) != tuple(shape) and t.numel() != int(np.prod(shape)):
        raise ValueError(f"{name}: expected shape {shape}, got {tuple(t.shape)}")
    return t


class Ctx:
    """An sdd_ctx handle with its grid shape."""

    def __init__(self, handle, nx, ny, sub_x, sub_y, stream):
        self.handle = handle
        self.nx, self.ny, self.sub_x, self.sub_y = nx, ny, sub_x, sub_y
        self.stream = stream

    def _check(self, st):
        if st != SDD_OK:
            msg = lib().sdd_last_error(self.handle)
            raise SddError(st, msg.decode() if msg else "")

    def __del__(self):
        try:
            sdd_destroy(self)
        except Exception:
            pass


def sdd_init(nx, ny=None, sub_x=1, sub_y=None, w=None, xi0=None, eta0=None, stream=None) -> Ctx:
    ny = nx if ny is None else ny
    sub_y = sub_x if sub_y is None else sub_y
    torch = _torch()
    for t, dt, name in ((w, torch.float32, "w"), (xi0, torch.float64, "xi0"), (eta0, torch.float64, "eta0")):
        if t is not None:
            _check_dev(t, dt, (ny, nx), name)
    h = ctypes.c_void_p()
    g = _Grid(nx, ny, sub_x, sub_y)
    st = lib().sdd_init(ctypes.byref(h), ctypes.byref(g), _ptr(w), _ptr(xi0), _ptr(eta0), _stream(stream))
    if st != SDD_OK:
        raise SddError(st, "sdd_init failed")
    return Ctx(h, nx, ny, sub_x, sub_y, stream)


def sdd_set_w(ctx: Ctx, w):
    _check_dev(w, _torch().float32, (ctx.ny, ctx.nx), "w")
    ctx._check(lib().sdd_set_w(ctx.handle, _ptr(w)))


def sdd_set_w_host(ctx: Ctx, w):
    """w: a CPU tensor (pinned for an asynchronous copy) or numpy float32 array."""
    if hasattr(w, "data_ptr"):
        assert w.dtype == _torch().float32 and w.is_contiguous() and w.numel() == ctx.nx * ctx.ny
        p = ctypes.c_void_p(w.data_ptr())
    else:
        w = np.ascontiguousarray(w, dtype=np.float32)
        p = ctypes.c_void_p(w.ctypes.data)
    ctx._check(lib().sdd_set_w_host(ctx.handle, p))


def sdd_set_fields(ctx: Ctx, xi, eta):
    torch = _torch()
    _check_dev(xi, torch.float64, (ctx.ny, ctx.nx), "xi")
    _check_dev(eta, torch.float64, (ctx.ny, ctx.nx), "eta")
    ctx._check(lib().sdd_set_fields(ctx.handle, _ptr(xi), _ptr(eta)))


def faces_len(nx, ny):
    return 2 * (2 * nx + 2 * ny)


def sdd_set_boundary(ctx: Ctx, faces=None):
    if faces is not None:
        _check_dev(faces, _torch().float64, (faces_len(ctx.nx, ctx.ny),), "faces")
    ctx._check(lib().sdd_set_boundary(ctx.handle, _ptr(faces)))


def sdd_get_faces(ctx: Ctx):
    torch = _torch()
    out = torch.empty(faces_len(ctx.nx, ctx.ny), dtype=torch.float64, device="cuda")
    ctx._check(lib().sdd_get_faces(ctx.handle, _ptr(out)))
    return out


def sdd_get_fields(ctx: Ctx):
    torch = _torch()
    xi = torch.empty((ctx.ny, ctx.nx), dtype=torch.float64, device="cuda")
    eta = torch.empty_like(xi)
    ctx._check(lib().sdd_get_fields(ctx.handle, _ptr(xi), _ptr(eta)))
    return xi, eta


def sdd_get_fields_host(ctx: Ctx):
    xi = np.empty((ctx.ny, ctx.nx), np.float64)
    eta = np.empty_like(xi)
    ctx._check(lib().sdd_get_fields_host(ctx.handle, ctypes.c_void_p(xi.ctypes.data), ctypes.c_void_p(eta.ctypes.data)))
    return xi, eta


def _nodes(x, y, n_paths):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    n = np.ascontiguousarray(np.broadcast_to(np.asarray(n_paths, dtype=np.int64), x.shape))
    keep = (x, y, n)
    return _Nodes(x.ctypes.data, y.ctypes.data, n.ctypes.data, x.size), keep


def _alloc_stats(count):
    torch = _torch()
    d = {k: torch.empty(count, dtype=torch.float64, device="cuda") for k in ("mean_xi", "mean_eta", "se_xi", "se_eta")}
    d["n_exit"] = torch.empty(count, dtype=torch.int64, device="cuda")
    d["path_steps"] = torch.empty(count, dtype=torch.int64, device="cuda")
    s = _Stats(*(d[k].data_ptr() for k in ("mean_xi", "mean_eta", "se_xi", "se_eta", "n_exit", "path_steps")))
    return d, s


def mc_params(dt, Dt, seed=0, step_index=0, exit_mode=0, block_threads=0, paths_per_task=0, node_word0=0,
              zero_map=0):
    return _McParams(dt, Dt, seed, step_index, exit_mode, block_threads, paths_per_task, node_word0, zero_map)


def sdd_interface_mc(ctx: Ctx, x, y, n_paths, dt, Dt, seed=0, step_index=0, exit_mode=0, block_threads=0,
                     paths_per_task=0, node_word0=0, zero_map=0, out=None):
    """Interface estimate at nodes (x, y) (host arrays). Returns a dict of cuda tensors."""
    nodes, keep = _nodes(x, y, n_paths)
    if out is None:
        out, s = _alloc_stats(nodes.count)
    else:
        s = _Stats(*(out[k].data_ptr() for k in ("mean_xi", "mean_eta", "se_xi", "se_eta", "n_exit", "path_steps")))
    p = mc_params(dt, Dt, seed, step_index, exit_mode, block_threads, paths_per_task, node_word0, zero_map)
    ctx._check(lib().sdd_interface_mc(ctx.handle, ctypes.byref(nodes), ctypes.byref(p), ctypes.byref(s)))
    del keep
    return out


def sdd_interface_mc_record(ctx: Ctx, x, y, n_paths, dt, Dt, seed=0, step_index=0, exit_mode=0, block_threads=0,
                            paths_per_task=0, node_word0=0, zero_map=0):
    """As sdd_interface_mc, plus per-path records (node after node)."""
    torch = _torch()
    nodes, keep = _nodes(x, y, n_paths)
    out, s = _alloc_stats(nodes.count)
    total = int(keep[2].sum())
    rec = {"steps": torch.empty(total, dtype=torch.int32, device="cuda"),
           "code": torch.empty(total, dtype=torch.int32, device="cuda")}
    for k in ("score_xi", "score_eta", "x_end", "y_end"):
        rec[k] = torch.empty(total, dtype=torch.float32, device="cuda")
    r = _Records(*(rec[k].data_ptr() for k in ("steps", "code", "score_xi", "score_eta", "x_end", "y_end")))
    p = mc_params(dt, Dt, seed, step_index, exit_mode, block_threads, paths_per_task, node_word0, zero_map)
    ctx._check(lib().sdd_interface_mc_record(ctx.handle, ctypes.byref(nodes), ctypes.byref(p), ctypes.byref(s),
                                             ctypes.byref(r)))
    del keep
    out.update(rec)
    return out


def sdd_interface_nodes(ctx: Ctx):
    n = ctypes.c_int64()
    ctx._check(lib().sdd_interface_nodes(ctx.handle, None, None, ctypes.byref(n)))
    x = np.empty(n.value)
    y = np.empty(n.value)
    ctx._check(lib().sdd_interface_nodes(ctx.handle, ctypes.c_void_p(x.ctypes.data), ctypes.c_void_p(y.ctypes.data),
                                         ctypes.byref(n)))
    return x, y


def sdd_subdomain_solve(ctx: Ctx, Dt, iface_xi, iface_eta, rtol=1e-12, max_iter=20000, want_iters=True):
    torch = _torch()
    xi = torch.empty((ctx.ny, ctx.nx), dtype=torch.float64, device="cuda")
    eta = torch.empty_like(xi)
    it = ctypes.c_int32(-1)
    st = lib().sdd_subdomain_solve(ctx.handle, Dt, _ptr(iface_xi), _ptr(iface_eta), rtol, max_iter, _ptr(xi),
                                   _ptr(eta), ctypes.byref(it) if want_iters else None)
    ctx._check(st)
    return xi, eta, it.value


def step_params(dt, Dt, seed=0, paths_per_node=10000, exit_mode=0, max_iter=20000, rtol=1e-12, tune=0):
    return _StepParams(dt, Dt, seed, paths_per_node, exit_mode, max_iter, rtol, tune, 0)


def sdd_step(ctx: Ctx, dt, Dt, seed=0, paths_per_node=10000, exit_mode=0, max_iter=20000, rtol=1e-12, tune=0):
    p = step_params(dt, Dt, seed, paths_per_node, exit_mode, max_iter, rtol, tune)
    ctx._check(lib().sdd_step(ctx.handle, ctypes.byref(p)))


def sdd_last_interface_stats(ctx: Ctx, out=None):
    """Interface statistics of the last sdd_step. `out`: optional dict of cuda or
    pinned host tensors (mean_xi, mean_eta, se_xi, se_eta float64; n_exit, path_steps int64)."""
    if out is None:
        n = ctypes.c_int64()
        ctx._check(lib().sdd_interface_nodes(ctx.handle, None, None, ctypes.byref(n)))
        out, s = _alloc_stats(n.value)
    else:
        s = _Stats(*(out[k].data_ptr() for k in ("mean_xi", "mean_eta", "se_xi", "se_eta", "n_exit", "path_steps")))
    ctx._check(lib().sdd_last_interface_stats(ctx.handle, ctypes.byref(s)))
    return out


def sdd_last_step_info(ctx: Ctx) -> dict:
    info = _StepInfo()
    ctx._check(lib().sdd_last_step_info(ctx.handle, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in _StepInfo._fields_}


def sdd_set_step_index(ctx: Ctx, n: int):
    ctx._check(lib().sdd_set_step_index(ctx.handle, n))


def sdd_get_step_index(ctx: Ctx) -> int:
    return int(lib().sdd_get_step_index(ctx.handle))


def sdd_set_pipeline(ctx: Ctx, on: bool):
    """Allow or forbid pipelined mesh steps (the solve beside the next step's paths)."""
    ctx._check(lib().sdd_set_pipeline(ctx.handle, 1 if on else 0))


def sdd_pipeline_in_use(ctx: Ctx) -> bool:
    return bool(lib().sdd_pipeline_in_use(ctx.handle))


def sdd_flush(ctx: Ctx):
    """Enqueue the pending iterations of the last pipelined step's solve."""
    ctx._check(lib().sdd_flush(ctx.handle))


def sdd_sync(ctx: Ctx):
    ctx._check(lib().sdd_sync(ctx.handle))


def sdd_last_error(ctx: Ctx) -> str:
    m = lib().sdd_last_error(ctx.handle)
    return m.decode() if m else ""


def sdd_destroy(ctx: Ctx):
    if ctx.handle is not None and ctx.handle.value:
        lib().sdd_destroy(ctx.handle)
    ctx.handle = ctypes.c_void_p(0)


def sdd_rng_draw(seed, counters, stream=None):
    """Philox words and unit normals for counters (n, 4) uint32 (cuda int32 tensor or numpy)."""
    torch = _torch()
    if isinstance(counters, np.ndarray):
        c = torch.from_numpy(np.ascontiguousarray(counters, dtype=np.uint32).view(np.int32)).cuda()
    else:
        c = counters.contiguous()
    n = c.numel() // 4
    words = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    normals = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    st = lib().sdd_rng_draw(seed, _ptr(c), n, _ptr(words), _ptr(normals), _stream(stream))
    if st != SDD_OK:
        raise SddError(st, "sdd_rng_draw failed")
    return words, normals


def sdd_interface_mc_static(w, xi, eta, x, y, n_paths, dt, Dt, seed=0, step_index=0, exit_mode=0, block_threads=0,
                            paths_per_task=0, node_word0=0, faces=None, out=None, stream=None, status=None):
    """The interface estimate without any allocation in the library (see include/sdd.h).

    w (float32), xi, eta (float64): cuda tensors of shape (ny, nx); x, y, n_paths: host arrays.
    `out`: optional dict of preallocated cuda tensors as returned by sdd_interface_mc.
    `status`: optional one-element int32 cuda tensor that receives the call's device status
    word on the stream (read it after synchronising); without it the call waits for the
    stream and raises SddError(SDD_EDEVICE) on a device error.
    """
    torch = _torch()
    ny, nx = w.shape
    _check_dev(w, torch.float32, (ny, nx), "w")
    _check_dev(xi, torch.float64, (ny, nx), "xi")
    _check_dev(eta, torch.float64, (ny, nx), "eta")
    if faces is not None:
        _check_dev(faces, torch.float64, (faces_len(nx, ny),), "faces")
    f = _Fields(nx, ny, w.data_ptr(), xi.data_ptr(), eta.data_ptr(), faces.data_ptr() if faces is not None else None)
    nodes, keep = _nodes(x, y, n_paths)
    if out is None:
        out, s = _alloc_stats(nodes.count)
    else:
        s = _Stats(*(out[k].data_ptr() for k in ("mean_xi", "mean_eta", "se_xi", "se_eta", "n_exit", "path_steps")))
    p = mc_params(dt, Dt, seed, step_index, exit_mode, block_threads, paths_per_task, node_word0)
    if status is not None:
        _check_dev(status, torch.int32, (1,), "status")
    st = lib().sdd_interface_mc_static(ctypes.byref(f), ctypes.byref(nodes), ctypes.byref(p), ctypes.byref(s),
                                       status.data_ptr() if status is not None else None, _stream(stream))
    del keep
    if st != SDD_OK:
        msg = {SDD_EINVAL: "sdd_interface_mc_static rejected its arguments",
               SDD_EDEVICE: "device error (w not finite and positive)"}.get(st, "CUDA error")
        raise SddError(st, msg)
    return out


def sdd_static_scratch_bytes() -> int:
    return int(lib().sdd_static_scratch_bytes())


class Batch:
    """An sdd_batch handle; keeps its contexts alive."""

    def __init__(self, handle, ctxs):
        self.handle = handle
        self.ctxs = list(ctxs)

    def _check(self, st):
        if st != SDD_OK:
            msg = lib().sdd_batch_last_error(self.handle)
            raise SddError(st, msg.decode() if msg else "")

    def __del__(self):
        try:
            sdd_batch_destroy(self)
        except Exception:
            pass


def sdd_batch_create(ctxs, stream=None) -> Batch:
    arr = (ctypes.c_void_p * len(ctxs))(*[c.handle.value for c in ctxs])
    h = ctypes.c_void_p()
    st = lib().sdd_batch_create(ctypes.byref(h), arr, len(ctxs), _stream(stream))
    if st != SDD_OK:
        raise SddError(st, "sdd_batch_create failed")
    return Batch(h, ctxs)


def sdd_batch_interface_mc(batch: Batch, node_lists, dt, Dt, seed=0, step_index=0, exit_mode=0, block_threads=0,
                           paths_per_task=0, node_word0=0):
    """node_lists: one (x, y, n_paths) per instance (host arrays). Returns one result dict per instance."""
    n = len(batch.ctxs)
    assert len(node_lists) == n
    keep, nodes, outs, stats = [], (_Nodes * n)(), [], (_Stats * n)()
    for k, (x, y, npaths) in enumerate(node_lists):
        nd, kp = _nodes(x, y, npaths)
        keep.append(kp)
        nodes[k] = nd
        o, s_ = _alloc_stats(nd.count)
        outs.append(o)
        stats[k] = s_
    p = mc_params(dt, Dt, seed, step_index, exit_mode, block_threads, paths_per_task, node_word0)
    batch._check(lib().sdd_batch_interface_mc(batch.handle, nodes, ctypes.byref(p), stats))
    del keep
    return outs


def sdd_batch_step(batch: Batch, dt, Dt, seed=0, paths_per_node=10000, exit_mode=0, max_iter=20000, rtol=1e-12,
                   tune=0):
    p = step_params(dt, Dt, seed, paths_per_node, exit_mode, max_iter, rtol, tune)
    batch._check(lib().sdd_batch_step(batch.handle, ctypes.byref(p)))


def sdd_batch_last_step_info(batch: Batch) -> dict:
    info = _StepInfo()
    batch._check(lib().sdd_batch_last_step_info(batch.handle, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in _StepInfo._fields_}


def sdd_batch_set_step_index(batch: Batch, n: int):
    batch._check(lib().sdd_batch_set_step_index(batch.handle, n))


def sdd_batch_sync(batch: Batch):
    batch._check(lib().sdd_batch_sync(batch.handle))


def sdd_batch_last_error(batch: Batch) -> str:
    m = lib().sdd_batch_last_error(batch.handle)
    return m.decode() if m else ""


def sdd_batch_destroy(batch: Batch):
    if batch.handle is not None and batch.handle.value:
        lib().sdd_batch_destroy(batch.handle)
    batch.handle = ctypes.c_void_p(0)


def sdd_autotune(ctx: Ctx, x, y, n_paths, dt, Dt, exit_mode=0) -> dict:
    """Pick the fastest launch shape for this node set (see include/sdd.h)."""
    nodes, keep = _nodes(x, y, n_paths)
    p = mc_params(dt, Dt, 0, 0, exit_mode, 0, 0)
    out = _Shape()
    ctx._check(lib().sdd_autotune(ctx.handle, ctypes.byref(nodes), ctypes.byref(p), ctypes.byref(out)))
    del keep
    return {"block_threads": out.block_threads, "paths_per_task": out.paths_per_task, "ms": out.ms,
            "zero_map": out.zero_map}


def sdd_batch_autotune(batch: Batch, node_lists, dt, Dt, exit_mode=0) -> dict:
    n = len(batch.ctxs)
    keep, nodes = [], (_Nodes * n)()
    for k, (x, y, npaths) in enumerate(node_lists):
        nd, kp = _nodes(x, y, npaths)
        keep.append(kp)
        nodes[k] = nd
    p = mc_params(dt, Dt, 0, 0, exit_mode, 0, 0)
    out = _Shape()
    batch._check(lib().sdd_batch_autotune(batch.handle, nodes, ctypes.byref(p), ctypes.byref(out)))
    del keep
    return {"block_threads": out.block_threads, "paths_per_task": out.paths_per_task, "ms": out.ms,
            "zero_map": out.zero_map}


def sdd_cv_set_table(ctx: Ctx, grad):
    """grad: cuda float64 tensor of shape (slices, ny, nx, 4) (see include/sdd.h)."""
    torch = _torch()
    if not (grad.is_cuda and grad.dtype == torch.float64 and grad.is_contiguous() and grad.dim() == 4
            and tuple(grad.shape[1:]) == (ctx.ny, ctx.nx, 4)):
        raise ValueError("grad: expected a contiguous cuda float64 tensor of shape (slices, ny, nx, 4)")
    ctx._check(lib().sdd_cv_set_table(ctx.handle, _ptr(grad), grad.shape[0]))


def sdd_cv_enable(ctx: Ctx, mode=SDD_CV_TABLE):
    """mode: SDD_CV_OFF / SDD_CV_TABLE / SDD_CV_MODEL / SDD_CV_FIELDS (True means SDD_CV_TABLE, False off)."""
    if mode is True:
        mode = SDD_CV_TABLE
    elif mode is False or mode is None:
        mode = SDD_CV_OFF
    ctx._check(lib().sdd_cv_enable(ctx.handle, int(mode)))


# ---------------------------------------------------------------- learned control variate

def _f32(t, n, name):
    torch = _torch()
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() >= n):
        raise ValueError(f"{name}: expected a contiguous cuda float32 tensor of at least {n} elements")
    return _ptr(t)


def sdd_mlp_init(ctx: Ctx, seed: int):
    """Initial parameter block (cuda float32, 2 * MLP_STRIDE)."""
    torch = _torch()
    th = torch.zeros(2 * MLP_STRIDE, dtype=torch.float32, device="cuda")
    ctx._check(lib().sdd_mlp_init(ctx.handle, seed, _ptr(th)))
    return th


def sdd_cv_samples(ctx: Ctx, per_horizon: int, *, dt: float, Dt: float, seed: int = 0, exit_mode: int = 0):
    """(feats (n, 5), targets (n, 2)) cuda float32 tensors, n = per_horizon * K."""
    torch = _torch()
    K = int(round(Dt / dt))
    n = per_horizon * K
    feats = torch.empty((n, MLP_INPUTS), dtype=torch.float32, device="cuda")
    targets = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    p = _SampleParams(per_horizon, exit_mode, dt, Dt, seed)
    ctx._check(lib().sdd_cv_samples(ctx.handle, ctypes.byref(p), _ptr(feats), _ptr(targets)))
    return feats, targets


def sdd_mlp_norm(ctx: Ctx, feats):
    torch = _torch()
    n = feats.shape[0]
    _f32(feats, n * MLP_INPUTS, "feats")
    norm = torch.zeros(2 * MLP_INPUTS, dtype=torch.float32, device="cuda")
    ctx._check(lib().sdd_mlp_norm(ctx.handle, _ptr(feats), n, _ptr(norm)))
    return norm


def sdd_mlp_grad(ctx: Ctx, theta, norm, feats, targets, rows=None):
    """(grad (2 * MLP_STRIDE), loss (2,)) of the mean squared error over the first rows."""
    torch = _torch()
    rows = feats.shape[0] if rows is None else rows
    _f32(theta, 2 * MLP_STRIDE, "theta")
    _f32(norm, 2 * MLP_INPUTS, "norm")
    _f32(feats, rows * MLP_INPUTS, "feats")
    _f32(targets, rows * 2, "targets")
    grad = torch.zeros(2 * MLP_STRIDE, dtype=torch.float32, device="cuda")
    loss = torch.zeros(2, dtype=torch.float32, device="cuda")
    ctx._check(lib().sdd_mlp_grad(ctx.handle, _ptr(theta), _ptr(norm), _ptr(feats), _ptr(targets), rows,
                                  _ptr(grad), _ptr(loss)))
    return grad, loss


def sdd_mlp_train(ctx: Ctx, theta, norm, feats, targets, *, epochs: int, batch: int, lr: float, max_steps: int = 0):
    """Adam in place on theta; returns the batch losses, shape (2, updates)."""
    torch = _torch()
    n = feats.shape[0]
    _f32(theta, 2 * MLP_STRIDE, "theta")
    _f32(norm, 2 * MLP_INPUTS, "norm")
    _f32(feats, n * MLP_INPUTS, "feats")
    _f32(targets, n * 2, "targets")
    total = epochs * (n // batch)
    steps = min(total, max_steps) if max_steps > 0 else total
    losses = torch.zeros((2, max(steps, 1)), dtype=torch.float32, device="cuda")
    p = _TrainParams(epochs, batch, lr, max_steps)
    ctx._check(lib().sdd_mlp_train(ctx.handle, _ptr(theta), _ptr(norm), _ptr(feats), _ptr(targets), n,
                                   ctypes.byref(p), _ptr(losses)))
    return losses[:, :steps]


def sdd_cv_tabulate(ctx: Ctx, theta, norm, slices: int, *, dt: float, Dt: float):
    _f32(theta, 2 * MLP_STRIDE, "theta")
    _f32(norm, 2 * MLP_INPUTS, "norm")
    ctx._check(lib().sdd_cv_tabulate(ctx.handle, _ptr(theta), _ptr(norm), slices, dt, Dt))


def sdd_cv_train(ctx: Ctx, *, per_horizon: int, dt: float, Dt: float, seed: int = 0, exit_mode: int = 0,
                 epochs: int = 20, batch: int = 4096, lr: float = 3e-3, max_steps: int = 0, slices: int = 0,
                 warm_start: bool = False, init_seed: int = 0):
    """Samples, training and tabulation in one call; returns the phase times and last losses."""
    p = _CvTrainParams(_SampleParams(per_horizon, exit_mode, dt, Dt, seed), _TrainParams(epochs, batch, lr, max_steps),
                       slices, 1 if warm_start else 0, init_seed)
    info = _CvTrainInfo()
    ctx._check(lib().sdd_cv_train(ctx.handle, ctypes.byref(p), ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in _CvTrainInfo._fields_}


def sdd_cv_get_model(ctx: Ctx):
    torch = _torch()
    th = torch.zeros(2 * MLP_STRIDE, dtype=torch.float32, device="cuda")
    norm = torch.zeros(2 * MLP_INPUTS, dtype=torch.float32, device="cuda")
    ctx._check(lib().sdd_cv_get_model(ctx.handle, _ptr(th), _ptr(norm)))
    return th, norm


def sdd_cv_losses(ctx: Ctx, count: int):
    torch = _torch()
    out = torch.zeros((2, max(count, 1)), dtype=torch.float32, device="cuda")
    ctx._check(lib().sdd_cv_losses(ctx.handle, _ptr(out), count))
    return out[:, :count]


def sdd_cv_get_table(ctx: Ctx, slices: int):
    """The context's current table, cuda float64 (slices, ny, nx, 4)."""
    torch = _torch()
    out = torch.zeros((slices, ctx.ny, ctx.nx, 4), dtype=torch.float64, device="cuda")
    ctx._check(lib().sdd_cv_get_table(ctx.handle, _ptr(out)))
    return out


def sdd_cv_set_fields_order(ctx: Ctx, order: int):
    """The binomial smoothing order of SDD_CV_FIELDS (odd 1..255; 0: by the grid)."""
    ctx._check(lib().sdd_cv_set_fields_order(ctx.handle, int(order)))


def sdd_cv_fields_order(ctx: Ctx) -> int:
    return int(lib().sdd_cv_fields_order(ctx.handle))


def sdd_cv_get_cells(ctx: Ctx):
    """SDD_CV_FIELDS's cell values from the current fields, cuda float32 (ny - 1, nx - 1, 4)."""
    torch = _torch()
    out = torch.zeros((ctx.ny - 1, ctx.nx - 1, 4), dtype=torch.float32, device="cuda")
    ctx._check(lib().sdd_cv_get_cells(ctx.handle, _ptr(out)))
    return out


def sdd_cv_set_model(ctx: Ctx, theta, norm, slices: int):
    _f32(theta, 2 * MLP_STRIDE, "theta")
    _f32(norm, 2 * MLP_INPUTS, "norm")
    ctx._check(lib().sdd_cv_set_model(ctx.handle, _ptr(theta), _ptr(norm), slices))


def sdd_set_solver(ctx: Ctx, solver: int):
    ctx._check(lib().sdd_set_solver(ctx.handle, int(solver)))


def sdd_solver_in_use(ctx: Ctx) -> int:
    return int(lib().sdd_solver_in_use(ctx.handle))


def sdd_set_keypoints(ctx: Ctx, on=True, spacing: int = 0):
    ctx._check(lib().sdd_set_keypoints(ctx.handle, 1 if on else 0, int(spacing)))


def sdd_keypoint_mask(ctx: Ctx):
    """Key-point mask of the current w: cuda uint8 tensor, one entry per interface node."""
    torch = _torch()
    n = len(sdd_interface_nodes(ctx)[0])
    out = torch.zeros(max(n, 1), dtype=torch.uint8, device="cuda")
    ctx._check(lib().sdd_keypoint_mask(ctx.handle, _ptr(out)))
    return out[:n]


def sdd_keypoint_fill(ctx: Ctx, mask, values_xi, values_eta):
    """The interface fill on given values: copies of values_* (one per interface node) whose entries
    outside `mask` are replaced by PCHIP along the interface lines (cuda float64 tensors)."""
    torch = _torch()
    n = len(sdd_interface_nodes(ctx)[0])
    m = torch.as_tensor(mask, device="cuda").to(torch.uint8).contiguous()
    vx = torch.as_tensor(values_xi, device="cuda", dtype=torch.float64).clone().contiguous()
    ve = torch.as_tensor(values_eta, device="cuda", dtype=torch.float64).clone().contiguous()
    if not (m.numel() == n and vx.numel() == n and ve.numel() == n):
        raise ValueError(f"mask and values: one entry per interface node ({n})")
    ctx._check(lib().sdd_keypoint_fill(ctx.handle, _ptr(m), _ptr(vx), _ptr(ve)))
    return vx, ve
