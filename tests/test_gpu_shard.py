"""Node sharding on the CUDA path, on one GPU: the ranks' node ranges run one
after the other in one process (no kernel waits on another), each with its
node words offset by its range's start (sdd_mc_params.node_word0). Their
results, put together, must be the whole list's estimate bit for bit, and a
mesh step made of them (the subdomain solve of the gathered values) must be the
unsharded step's.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sdd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1402_0266_gb300 import build
    build.build()
    import paper_1402_0266_gb300 as m
    return m


def _ctx(sdd, n, t):
    import torch
    X, Y = W.identity_fields(n)
    return sdd.sdd_init(n, n, 2, 2, w=torch.from_numpy(W.w_front(n, t)).cuda(), xi0=torch.from_numpy(X).cuda(),
                        eta0=torch.from_numpy(Y).cuda())


def _np(d):
    return {k: v.cpu().numpy() for k, v in d.items()}


def test_node_ranges_with_offset_words_equal_the_whole_list(sdd):
    from paper_1402_0266_gb300 import shard
    n = 129
    ctx = _ctx(sdd, n, 0.2)
    xs, ys = sdd.sdd_interface_nodes(ctx)
    npaths = np.where(np.arange(xs.size) % 5 == 0, 3000, 1100)
    kw = dict(dt=1e-4, Dt=1e-2, seed=4, step_index=3, paths_per_task=256)
    whole = _np(sdd.sdd_interface_mc(ctx, xs, ys, npaths, **kw))
    for world in (2, 3, 8):
        parts = [_np(sdd.sdd_interface_mc(ctx, xs[lo:hi], ys[lo:hi], npaths[lo:hi], node_word0=lo, **kw))
                 for lo, hi in shard.node_ranges(npaths, world)]
        for k in whole:
            np.testing.assert_array_equal(np.concatenate([p[k] for p in parts]), whole[k], err_msg=f"{world} {k}")
    # without the offset the ranges would draw other streams
    lo, hi = shard.node_ranges(npaths, 2)[1]
    other = _np(sdd.sdd_interface_mc(ctx, xs[lo:hi], ys[lo:hi], npaths[lo:hi], **kw))
    assert not np.array_equal(other["mean_xi"], whole["mean_xi"][lo:hi])


def test_sharded_mesh_step_equals_the_unsharded_step(sdd):
    import torch
    from paper_1402_0266_gb300 import shard
    n = 129
    a = _ctx(sdd, n, 0.1)
    b = _ctx(sdd, n, 0.1)
    kw = dict(dt=1e-4, Dt=1e-2, seed=8, paths_per_node=2000, paths_per_task=256)
    for step in range(2):
        w = torch.from_numpy(W.w_front(n, 0.1 + 0.01 * step)).cuda()
        sdd.sdd_set_w(a, w)
        sdd.sdd_set_w(b, w)
        # one rank's view of a two-rank step, with both ranges estimated here in turn
        xs, ys = sdd.sdd_interface_nodes(a)
        stats = shard.sharded_estimate(
            lambda x, y, p, w0: sdd.sdd_interface_mc(a, x, y, p, dt=kw["dt"], Dt=kw["Dt"], seed=kw["seed"],
                                                     step_index=sdd.sdd_get_step_index(a),
                                                     paths_per_task=kw["paths_per_task"], node_word0=w0),
            xs, ys, kw["paths_per_node"], 0, 1)
        xi, eta, _ = sdd.sdd_subdomain_solve(a, kw["Dt"], stats["mean_xi"], stats["mean_eta"])
        sdd.sdd_set_fields(a, xi, eta)
        sdd.sdd_set_step_index(a, sdd.sdd_get_step_index(a) + 1)
        # the library's own sharded step with one rank
        sb = shard.sdd_sharded_step(b, rank=0, world=1, **kw)
        for k in stats:
            np.testing.assert_array_equal(stats[k].cpu().numpy(), sb[k].cpu().numpy())
        fa = [f.cpu().numpy() for f in sdd.sdd_get_fields(a)]
        fb = [f.cpu().numpy() for f in sdd.sdd_get_fields(b)]
        np.testing.assert_array_equal(fa[0], fb[0])
        np.testing.assert_array_equal(fa[1], fb[1])
        assert sdd.sdd_get_step_index(b) == step + 1
