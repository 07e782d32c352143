"""The allocation-free entry point against the regular one.

sdd_interface_mc_static serves callers that may not allocate device memory
while they run (a real-time loop, a host with a fixed memory pool, a plugin
handed only pointers and a stream): it keeps all of its working memory in one
static device array. This file checks, through the C ABI, that it returns
what sdd_interface_mc returns for the same inputs, on two calls in a row (the
second one reuses the array left behind by the first). It is named so that
pytest collects it last.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("mean_xi", "mean_eta", "se_xi", "se_eta", "n_exit", "path_steps")


@pytest.fixture(scope="module")
def sdd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1402_0266_gb300 import build
    build.build()
    import paper_1402_0266_gb300 as m
    return m


def _np(d):
    return {k: d[k].cpu().numpy() for k in KEYS}


def _cases():
    n = 65
    w = W.w_front(n, 0.25)
    X, Y = W.grid(n)
    xi0 = X + 0.02 * np.sin(np.pi * X) * np.sin(np.pi * Y)
    eta0 = Y.copy()
    xs, ys = W.interface_node_coords(n, n, 2, 2)
    xs = np.concatenate([xs, [0.0, 0.5, 0.013]])
    ys = np.concatenate([ys, [0.4, 1.0, 0.77]])
    npaths = np.full(xs.size, 1500)
    npaths[::7] = 37
    return n, w, xi0, eta0, xs, ys, npaths


@pytest.mark.parametrize("exit_mode,user_faces", [(0, False), (1, True)])
def test_static_entry_point_matches_regular_entry_point(sdd, exit_mode, user_faces):
    import torch
    n, w, xi0, eta0, xs, ys, npaths = _cases()
    wt = torch.from_numpy(w).cuda()
    xt = torch.from_numpy(xi0).cuda()
    et = torch.from_numpy(eta0).cuda()
    faces = None
    if user_faces:
        rng = np.random.default_rng(4)
        faces = torch.from_numpy(rng.uniform(0.0, 1.0, size=sdd.faces_len(n, n))).cuda()
    ctx = sdd.sdd_init(n, n, 2, 2, w=wt, xi0=xt, eta0=et)
    if faces is not None:
        sdd.sdd_set_boundary(ctx, faces)
    kw = dict(dt=1e-4, Dt=1e-2, seed=11, step_index=4, exit_mode=exit_mode, paths_per_task=128)
    ref = _np(sdd.sdd_interface_mc(ctx, xs, ys, npaths, **kw))
    sdd.sdd_sync(ctx)
    for call in range(2):
        got = sdd.sdd_interface_mc_static(wt, xt, et, xs, ys, npaths, faces=faces, **kw)
        torch.cuda.synchronize()
        got = _np(got)
        for k in ("mean_xi", "mean_eta", "se_xi", "se_eta"):
            np.testing.assert_allclose(got[k], ref[k], rtol=0, atol=1e-12, err_msg=f"call {call}: {k}")
        np.testing.assert_array_equal(got["n_exit"], ref["n_exit"])
        np.testing.assert_array_equal(got["path_steps"], ref["path_steps"])


def test_static_entry_point_rejects_sizes_beyond_its_limits(sdd):
    import torch
    n = 259  # above the 257 x 257 limit
    w = torch.ones((n, n), dtype=torch.float32, device="cuda")
    f = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_interface_mc_static(w, f, f, [0.5], [0.5], [10], dt=1e-3, Dt=1e-2)
    assert e.value.status == sdd.SDD_EINVAL
    n = 17
    w = torch.ones((n, n), dtype=torch.float32, device="cuda")
    f = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    with pytest.raises(sdd.SddError):  # more nodes than the static node list holds
        sdd.sdd_interface_mc_static(w, f, f, np.full(9000, 0.5), np.full(9000, 0.5), 10, dt=1e-3, Dt=1e-2)
    assert sdd.sdd_static_scratch_bytes() < 16 * 2 ** 20


def test_static_entry_point_reports_device_errors(sdd):
    # a w that is not positive at one node is a device-side error: reported by the call
    # itself (it waits for the stream) or, when the caller gives a device word, in that word;
    # the next clean call reports none
    import torch
    n = 17
    X, Y = W.identity_fields(n)
    xi = torch.from_numpy(X).cuda()
    eta = torch.from_numpy(Y).cuda()
    bad = torch.ones((n, n), dtype=torch.float32, device="cuda")
    bad[5, 7] = 0.0
    good = torch.ones((n, n), dtype=torch.float32, device="cuda")
    kw = dict(dt=1e-3, Dt=1e-2, seed=3)
    with pytest.raises(sdd.SddError) as e:
        sdd.sdd_interface_mc_static(bad, xi, eta, [0.5], [0.5], [100], **kw)
    assert e.value.status == sdd.SDD_EDEVICE
    sdd.sdd_interface_mc_static(good, xi, eta, [0.5], [0.5], [100], **kw)
    word = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    sdd.sdd_interface_mc_static(bad, xi, eta, [0.5], [0.5], [100], status=word, **kw)
    torch.cuda.synchronize()
    assert int(word.item()) != 0
    out = sdd.sdd_interface_mc_static(good, xi, eta, [0.5], [0.5], [100], status=word, **kw)
    torch.cuda.synchronize()
    assert int(word.item()) == 0
    assert abs(float(out["mean_xi"].item()) - 0.5) < 0.05
