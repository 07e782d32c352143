"""Batched instances (one persistent launch) against the oracle on the same streams."""
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


def _np(d):
    return {k: v.cpu().numpy() for k, v in d.items()}


def _ctx(sdd, w, xi0, eta0, sub):
    import torch
    ny, nx = w.shape
    return sdd.sdd_init(nx, ny, sub, sub, w=torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda(),
                        xi0=torch.from_numpy(np.ascontiguousarray(xi0)).cuda(),
                        eta0=torch.from_numpy(np.ascontiguousarray(eta0)).cuda())


def _assert_close(g, o, what):
    for f in ("xi", "eta"):
        d = np.abs(g["mean_" + f] - o["mean_" + f])
        assert np.all(d <= 3 * o["se_" + f] + 1e-4), (what, f, d.max())
        assert np.median(d) <= 1e-5, (what, f, np.median(d))


def test_batch_estimate_matches_oracle(sdd, oracle_mod):
    specs = [(33, W.w_smooth_random(33, 1), 2), (65, W.w_front(65, 0.2), 2), (129, W.w_bump(129, 0.4, 0.6, 0.1, 8.0), 2),
             (65, W.w_ring(65, 0.1), 4)]
    ctxs, probs, lists = [], [], []
    rng = np.random.default_rng(0)
    for n, w, sub in specs:
        xi0, eta0 = W.identity_fields(n)
        ctxs.append(_ctx(sdd, w, xi0, eta0, sub))
        probs.append(oracle_mod.Problem(w, xi0, eta0))
        xs, ys = W.interface_node_coords(n, n, sub, sub)
        pick = np.unique(rng.integers(0, xs.size, size=12))
        xs = np.concatenate([xs[pick], [0.0, 0.31]])
        ys = np.concatenate([ys[pick], [0.5, 0.002]])
        npaths = rng.integers(1, 1500, size=xs.size)
        lists.append((xs, ys, npaths))
    batch = sdd.sdd_batch_create(ctxs)
    kw = dict(dt=1e-4, Dt=5e-3, seed=42, step_index=3)
    outs = [_np(o) for o in sdd.sdd_batch_interface_mc(batch, lists, **kw)]
    sdd.sdd_batch_sync(batch)
    offset = 0
    for k, ((xs, ys, npaths), P) in enumerate(zip(lists, probs)):
        o = oracle_mod.interface_mc(P, xs, ys, npaths, node_ids=np.arange(xs.size, dtype=np.uint32) + offset, **kw)
        _assert_close(outs[k], o, f"instance {k}")
        np.testing.assert_array_equal(outs[k]["path_steps"] > 0, o["path_steps"] > 0)
        offset += xs.size
    # instance 0 numbers its nodes from 0, as a context of its own does: identical results
    single = _np(sdd.sdd_interface_mc(ctxs[0], *lists[0], **kw))
    for key in ("mean_xi", "mean_eta", "n_exit", "path_steps"):
        np.testing.assert_allclose(single[key], outs[0][key], rtol=0, atol=1e-8)


def test_batch_steps_match_oracle(sdd, oracle_mod):
    import torch
    specs = [(33, 2), (65, 2), (41, 3)]
    dt, Dt, paths = 1e-4, 1e-2, 1500
    ctxs, state = [], []
    for n, sub in specs:
        xi0, eta0 = W.identity_fields(n)
        ctxs.append(_ctx(sdd, W.w_front(n, 0.0), xi0, eta0, sub))
        state.append([xi0, eta0])
    batch = sdd.sdd_batch_create(ctxs)
    for step in range(2):
        for c, (n, sub) in zip(ctxs, specs):
            sdd.sdd_set_w(c, torch.from_numpy(W.w_front(n, step * Dt)).cuda())
        sdd.sdd_batch_step(batch, dt=dt, Dt=Dt, seed=9, paths_per_node=paths, rtol=1e-13, max_iter=50000)
        sdd.sdd_batch_sync(batch)
        offset = 0
        for k, (c, (n, sub)) in enumerate(zip(ctxs, specs)):
            g = _np(sdd.sdd_last_interface_stats(c))
            ii, jj = W.interface_nodes(n, n, sub, sub)
            new, o = oracle_mod.dd_step(W.w_front(n, step * Dt), state[k][0], state[k][1], sub_x=sub, sub_y=sub,
                                        dt=dt, Dt=Dt, n_paths=paths, seed=9, step_index=step, nodes_ij=(ii, jj),
                                        node_word0=offset)
            if step == 0:
                _assert_close(g, o, f"instance {k} step {step}")
                gx, ge = (a.cpu().numpy() for a in sdd.sdd_get_fields(c))
                gap = max(np.abs(gx - new[0]).max(), np.abs(ge - new[1]).max())
                iface_gap = max(np.abs(g["mean_xi"] - o["mean_xi"]).max(), np.abs(g["mean_eta"] - o["mean_eta"]).max())
                assert gap <= iface_gap + 1e-9
            state[k] = new
            offset += ii.size
    info = sdd.sdd_batch_last_step_info(batch)
    assert info["kernel_nodes"] > 0 and info["paths_ms"] > 0
    assert sdd.sdd_get_step_index(ctxs[0]) == 2


def test_batch64_workload_sampled_parity(sdd, oracle_mod):
    # the 64-instance workload in one launch; the oracle recomputes a sample of nodes path by
    # path: each sampled node is run again on its own context with the node word the batch gave
    # it (sdd_mc_params.node_word0) and the same task size, which must reproduce the batch's
    # results bit for bit, and its per-path records are compared with the oracle's
    from tests import _parity as PT
    insts = W.batch64_instances(seed=0)
    ctxs, lists, probs = [], [], []
    for I in insts:
        w = W.w_bump(I.n, I.cx, I.cy, I.width, I.alpha)
        xi0, eta0 = W.identity_fields(I.n)
        ctxs.append(_ctx(sdd, w, xi0, eta0, 2))
        xs, ys = I.nodes_i / (I.n - 1), I.nodes_j / (I.n - 1)
        lists.append((xs, ys, I.paths))
        probs.append((w, xi0, eta0))
    batch = sdd.sdd_batch_create(ctxs)
    kw = dict(dt=1e-4, Dt=1e-2, seed=0)
    outs = [_np(o) for o in sdd.sdd_batch_interface_mc(batch, lists, paths_per_task=256, **kw)]
    sdd.sdd_batch_sync(batch)
    offsets = np.concatenate([[0], np.cumsum([l[0].size for l in lists])])
    checked = 0
    for k in (0, 17, 40, 63):
        xs, ys, npaths = lists[k]
        pick = np.array([0, xs.size // 2, xs.size - 1])
        P = oracle_mod.Problem(*probs[k])
        for p in pick:
            word = int(offsets[k] + p)
            r = _np(sdd.sdd_interface_mc_record(ctxs[k], xs[p:p + 1], ys[p:p + 1], npaths[p:p + 1],
                                                paths_per_task=256, node_word0=word, **kw))
            for key in ("mean_xi", "mean_eta", "se_xi", "se_eta", "n_exit", "path_steps"):
                np.testing.assert_array_equal(r[key][0], outs[k][key][p], err_msg=f"{k} {p} {key}")
            o = oracle_mod.interface_mc(P, xs[p:p + 1], ys[p:p + 1], npaths[p:p + 1],
                                        node_ids=np.array([word], np.uint32), record=True, **kw)
            same, rep = PT.assert_records(r, o)
            PT.assert_flips_near_boundary(oracle_mod, P, xs[p:p + 1], ys[p:p + 1], npaths[p:p + 1], r, o, same,
                                          node_ids=np.array([word], np.uint32), **kw)
            PT.assert_nodes(r, o, npaths[p:p + 1], same, np.array([0, npaths[p]]))
            checked += int(npaths[p])
    assert checked > 10 ** 5
    for o in outs:
        assert np.all((o["mean_xi"] >= 0) & (o["mean_xi"] <= 1))
