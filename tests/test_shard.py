"""Node sharding of the interface estimate (Sec. 4, "fully parallel"): the
partition, the node-word offsets and the all-gather of the per-node results,
on two gloo ranks on the host (127.0.0.1), with the FP64 oracle as the
estimate of each rank's node range. A sharded estimate and a sharded mesh step
must equal the single-rank ones bit for bit.
"""
import os
import socket

import numpy as np
import pytest

import workloads as W


def test_node_ranges_cover_the_list_and_balance_the_paths():
    from paper_1402_0266_gb300 import shard
    rng = np.random.default_rng(3)
    for n, world in ((509, 2), (509, 8), (7, 4), (3, 8), (0, 2), (1000, 3)):
        npaths = rng.integers(1, 5000, size=n)
        r = shard.node_ranges(npaths, world)
        assert len(r) == world and r[0][0] == 0 and r[-1][1] == n
        for (a, b), (c, d) in zip(r, r[1:]):
            assert b == c and a <= b
        if n:
            share = npaths.sum() / world
            for lo, hi in r:
                assert abs(int(npaths[lo:hi].sum()) - share) <= npaths.max()
    assert shard.node_ranges([5, 5, 5, 5], 2) == [(0, 2), (2, 4)]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import oracle
    oracle.build()
    n = 33
    w = W.w_front(n, 0.2).astype(np.float64)
    xi0, eta0 = W.identity_fields(n)
    return oracle, n, w, xi0, eta0


def _oracle_estimate(oracle, P, dt, Dt, seed, step):
    import torch

    def est(x, y, npaths, word0):
        r = oracle.interface_mc(P, x, y, npaths, dt=dt, Dt=Dt, seed=seed, step_index=step,
                                node_ids=np.arange(x.size, dtype=np.uint32) + np.uint32(word0), threads=2)
        return {k: torch.from_numpy(np.asarray(r[k])) for k in ("mean_xi", "mean_eta", "se_xi", "se_eta", "n_exit",
                                                                "path_steps")}
    return est


def _worker(rank, port, q):
    os.environ.update(WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist

    from paper_1402_0266_gb300 import shard
    dist.init_process_group("gloo")
    oracle, n, w, xi0, eta0 = _problem()
    from oracle import solver
    dt, Dt = 1e-3, 2e-2
    ii, jj = W.interface_nodes(n, n, 2, 2)
    xs, ys = ii / (n - 1), jj / (n - 1)
    npaths = np.where(np.arange(xs.size) % 3 == 0, 300, 170)
    P = oracle.Problem(w, xi0, eta0)
    # the sharded estimate
    est = shard.sharded_estimate(_oracle_estimate(oracle, P, dt, Dt, 5, 1), xs, ys, npaths, rank, 2)
    est = {k: v.numpy() for k, v in est.items()}
    # a sharded mesh step: the gathered interface values into the same subdomain solves on every rank
    bx = oracle.boundary_grid(P.faces, n, n, 0, P.xi0)
    be = oracle.boundary_grid(P.faces, n, n, 1, P.eta0)
    bx[jj, ii] = est["mean_xi"]
    be[jj, ii] = est["mean_eta"]
    fields = solver.subdomain_solve(P.w, [P.xi0, P.eta0], [bx, be], 2, 2, Dt)
    q.put((rank, est, fields, shard.node_ranges(npaths, 2)[rank]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_estimate_and_the_mesh_step_bit_for_bit():
    pytest.importorskip("torch.distributed")
    import torch.multiprocessing as mp
    oracle, n, w, xi0, eta0 = _problem()
    dt, Dt = 1e-3, 2e-2
    ii, jj = W.interface_nodes(n, n, 2, 2)
    xs, ys = ii / (n - 1), jj / (n - 1)
    npaths = np.where(np.arange(xs.size) % 3 == 0, 300, 170)
    P = oracle.Problem(w, xi0, eta0)
    whole = oracle.interface_mc(P, xs, ys, npaths, dt=dt, Dt=Dt, seed=5, step_index=1)
    new, r = oracle.dd_step(w, xi0, eta0, sub_x=2, sub_y=2, dt=dt, Dt=Dt, n_paths=npaths, seed=5, step_index=1,
                            nodes_ij=(ii, jj))

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(k, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (lo0, hi0), (lo1, hi1) = res[0][3], res[1][3]
    assert lo0 == 0 and hi0 == lo1 and hi1 == xs.size and 0 < hi0 < xs.size
    for rank, est, fields, _ in res:
        for k in ("mean_xi", "mean_eta", "se_xi", "se_eta", "n_exit", "path_steps"):
            np.testing.assert_array_equal(est[k], whole[k], err_msg=f"rank {rank} {k}")
        np.testing.assert_array_equal(fields[0], new[0])
        np.testing.assert_array_equal(fields[1], new[1])
