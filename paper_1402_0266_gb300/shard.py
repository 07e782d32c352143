"""Node sharding of the interface estimate over ranks, one process per GPU.

Sec. 4 ("the method is fully parallel"): the paths, and so the interface
nodes, are independent; the only exchange of a mesh step is the interface
values that the deterministic subdomain solves need. Here each rank takes one
contiguous range of the interface nodes, the ranges weighted by path count;
estimates it with the node words of its Philox counters offset by the range's
first index (sdd_mc_params.node_word0), so that at a fixed paths_per_task every
node's results are those of a single-rank estimate of the whole list, bit for
bit; the per-node results are then all-gathered (NCCL between GPUs, gloo
between host processes), and every rank runs the same subdomain solve on the
same interface values and so keeps the same fields.

Only the estimate is split: the solve is repeated on every rank (it is a few
percent of a mesh step at 2049 x 2049, 8 x 8 subdomains), which keeps the
exchange to the per-node results (6 numbers per node).

The functions take the estimate and the solve as callables so that the same
partition and exchange run on the CUDA path (sdd_sharded_step) and on any
other implementation of the estimate with the same node numbering.
"""
from __future__ import annotations

import numpy as np

# the per-node results of an estimate, in the order they are exchanged
STAT_KEYS = ("mean_xi", "mean_eta", "se_xi", "se_eta", "n_exit", "path_steps")


def node_ranges(n_paths, world: int):
    """Contiguous node ranges [lo, hi), one per rank, in rank order: range r ends
    where the running path count first reaches (r + 1) / world of the total, so
    every range's path count is within one node's of the even share."""
    n_paths = np.asarray(n_paths, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    n = n_paths.size
    cum = np.cumsum(n_paths)
    total = int(cum[-1]) if n else 0
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        k = int(np.searchsorted(cum, target, side="left")) + 1 if n else 0
        bounds.append(min(max(k, bounds[-1]), n))
    bounds.append(n)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def _backend_device(group=None):
    import torch.distributed as dist
    return "cuda" if dist.get_backend(group) == "nccl" else "cpu"


def gather_node_results(local: dict, ranges, group=None) -> dict:
    """All-gather every rank's per-node results (STAT_KEYS, one entry per node of
    its range) into the whole list's arrays, in rank order. Returns tensors on
    the device of this rank's results."""
    import torch
    import torch.distributed as dist
    world = len(ranges)
    most = max(hi - lo for lo, hi in ranges)
    dev = _backend_device(group)
    out = {}
    for key in STAT_KEYS:
        v = local[key]
        home = v.device
        v = v.to(dev)
        buf = torch.zeros(most, dtype=v.dtype, device=dev)
        buf[:v.numel()] = v
        parts = [torch.empty_like(buf) for _ in range(world)]
        dist.all_gather(parts, buf, group=group)
        out[key] = torch.cat([parts[r][:hi - lo] for r, (lo, hi) in enumerate(ranges)]).to(home)
    return out


def sharded_estimate(estimate, xs, ys, n_paths, rank: int, world: int, group=None):
    """This rank's share of the interface estimate, then the whole list's results.

    estimate(x, y, n_paths, node_word0) -> dict of STAT_KEYS tensors for one
    contiguous node range whose first node has node word node_word0."""
    xs = np.asarray(xs, dtype=np.float64)
    ys = np.asarray(ys, dtype=np.float64)
    n_paths = np.broadcast_to(np.asarray(n_paths, dtype=np.int64), xs.shape).copy()
    ranges = node_ranges(n_paths, world)
    lo, hi = ranges[rank]
    local = estimate(xs[lo:hi], ys[lo:hi], n_paths[lo:hi], lo)
    if world == 1:
        return local
    return gather_node_results(local, ranges, group)


def sdd_sharded_step(ctx, *, dt, Dt, seed, paths_per_node, paths_per_task, rank, world, group=None,
                     exit_mode=0, rtol=1e-12, max_iter=20000):
    """One mesh step t_{n-1} -> t_n of a context, its interface estimate split over
    the ranks: this rank's node range (step index n = the context's, node words
    offset by the range's start), the all-gather of the per-node results, the
    subdomain solves with the gathered interface values (every rank the same),
    the new fields and step index into the context. paths_per_task must be given
    (the node results depend on the task size at the last bits of the sums).
    Returns the whole list's interface statistics (cuda tensors)."""
    import paper_1402_0266_gb300 as sdd
    if paths_per_task <= 0:
        raise ValueError("sdd_sharded_step needs an explicit paths_per_task")
    xs, ys = sdd.sdd_interface_nodes(ctx)
    n = sdd.sdd_get_step_index(ctx)

    def estimate(x, y, npaths, word0):
        return sdd.sdd_interface_mc(ctx, x, y, npaths, dt=dt, Dt=Dt, seed=seed, step_index=n, exit_mode=exit_mode,
                                    paths_per_task=paths_per_task, node_word0=word0)

    stats = sharded_estimate(estimate, xs, ys, np.full(xs.size, paths_per_node, dtype=np.int64), rank, world, group)
    xi, eta, _ = sdd.sdd_subdomain_solve(ctx, Dt, stats["mean_xi"], stats["mean_eta"], rtol=rtol, max_iter=max_iter)
    sdd.sdd_set_fields(ctx, xi, eta)
    sdd.sdd_set_step_index(ctx, n + 1)
    return stats
