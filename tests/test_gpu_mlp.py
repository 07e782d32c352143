"""The learned control variate on the GPU against the oracle's FP64 network.

Initial weights and training-sample start points are bit-identical (same
Philox words, same rounding); single-path scores agree like every other path
record; the FP32 gradient agrees with FP64 backpropagation to FP32 rounding;
Adam's first updates agree; the BF16 tensor-core table agrees with the FP64
forward-mode derivative within the error of BF16 operands; and a network
trained by the GPU cuts the variance of the estimator while leaving its mean.
"""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

STRIDE = 4616
P = 4609


@pytest.fixture(scope="module")
def sdd():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1402_0266_gb300 import build
    build.build()
    import paper_1402_0266_gb300 as m
    return m


@pytest.fixture(scope="module")
def mlp(oracle_mod):
    from oracle import mlp as m
    return m


def _ctx(sdd, w, xi0, eta0, sub=2, faces=None):
    import torch
    ny, nx = w.shape
    ctx = sdd.sdd_init(nx, ny, sub, sub, w=torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda(),
                       xi0=torch.from_numpy(np.ascontiguousarray(xi0)).cuda(),
                       eta0=torch.from_numpy(np.ascontiguousarray(eta0)).cuda())
    if faces is not None:
        sdd.sdd_set_boundary(ctx, torch.from_numpy(np.ascontiguousarray(faces, np.float64)).cuda())
    return ctx


def _heat(oracle_mod, sdd):
    xi0, eta0 = W.heat65_fields()
    faces = np.zeros(oracle_mod.faces_len(65, 65))
    P_ = oracle_mod.Problem(W.w_const(65), xi0, eta0, faces)
    return P_, _ctx(sdd, W.w_const(65), xi0, eta0, faces=faces)


def _front(oracle_mod, sdd, n=65):
    w = W.w_front(n, 0.15).astype(np.float32).astype(np.float64)
    xi0, eta0 = W.identity_fields(n)
    return oracle_mod.Problem(w, xi0, eta0), _ctx(sdd, w, xi0, eta0)


def _oracle_rows(mlp, Pr, per_horizon, seed):
    """Training rows from the oracle's own samples of the method, as the GPU kernels take them
    (single precision), on the device and as the FP64 values of those single-precision numbers."""
    import torch
    F, Y = mlp.training_samples(Pr, per_horizon=per_horizon, dt=1e-3, Dt=1e-2, seed=seed)
    F32, Y32 = np.ascontiguousarray(F, np.float32), np.ascontiguousarray(Y, np.float32)
    return (torch.from_numpy(F32).cuda(), torch.from_numpy(Y32).cuda(), F32.astype(np.float64),
            Y32.astype(np.float64))


def _oracle_norm(mlp, F):
    """The oracle's standardisation of rows F: (mu, 1 / sd) in single precision, on the device and
    as FP64 values."""
    import torch
    mu, s = mlp.standardise(F)
    nv = np.concatenate([mu, s]).astype(np.float32)
    return torch.from_numpy(nv).cuda(), nv.astype(np.float64)


def _split(theta):
    t = theta.cpu().numpy().astype(np.float64)
    return np.stack([t[:P], t[STRIDE:STRIDE + P]])


def test_initial_weights_bit_identical(sdd, mlp, oracle_mod):
    _, ctx = _front(oracle_mod, sdd, 17)
    for seed in (0, 7, 2 ** 64 - 1):
        th = sdd.sdd_mlp_init(ctx, seed).cpu().numpy()
        want = mlp.init_params(seed)
        np.testing.assert_array_equal(th[:P], want[0].astype(np.float32))
        np.testing.assert_array_equal(th[STRIDE:STRIDE + P], want[1].astype(np.float32))
        assert np.all(th[P:STRIDE] == 0) and np.all(th[STRIDE + P:] == 0)


@pytest.mark.parametrize("exit_mode", [0, 1])
def test_training_samples_match_oracle(sdd, mlp, oracle_mod, exit_mode):
    Pr, ctx = _front(oracle_mod, sdd)
    M, dt, Dt = 300, 1e-3, 1e-2
    feats, targets = sdd.sdd_cv_samples(ctx, M, dt=dt, Dt=Dt, seed=5, exit_mode=exit_mode)
    F, Y = mlp.training_samples(Pr, per_horizon=M, dt=dt, Dt=Dt, seed=5, exit_mode=exit_mode)
    g = feats.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(g[:, :3], F[:, :3].astype(np.float32))    # starts and times: same bits
    np.testing.assert_allclose(g[:, 3:], F[:, 3:], rtol=2e-6, atol=1e-6)    # w, r interpolated in FP32 tables
    d = np.abs(targets.cpu().numpy().astype(np.float64) - Y)
    same = (d <= 1e-4).all(axis=1)
    assert same.mean() >= 0.995, same.mean()    # the records' tolerance: exit decisions on the same streams


def test_standardisation_matches_oracle(sdd, mlp, oracle_mod):
    Pr, ctx = _front(oracle_mod, sdd)
    feats, _, F, _ = _oracle_rows(mlp, Pr, 500, 1)
    norm = sdd.sdd_mlp_norm(ctx, feats).cpu().numpy().astype(np.float64)
    mu, s = mlp.standardise(F)
    np.testing.assert_allclose(norm[:5], mu, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(norm[5:], s, rtol=1e-5)


def _random_model(sdd, ctx, mlp, seed, scale=0.3):
    import torch
    th = mlp.init_params(seed)
    rng = np.random.default_rng(seed)
    th = th + scale * rng.normal(size=th.shape)          # biases and weights away from the initial values
    block = np.zeros(2 * STRIDE, np.float32)
    block[:P] = th[0]
    block[STRIDE:STRIDE + P] = th[1]
    return torch.from_numpy(block).cuda()


def test_gradient_matches_oracle_backprop(sdd, mlp, oracle_mod):
    Pr, ctx = _front(oracle_mod, sdd)
    feats, targets, F, Yall = _oracle_rows(mlp, Pr, 240, 2)                    # 2400 rows
    norm, nv = _oracle_norm(mlp, F)
    theta = _random_model(sdd, ctx, mlp, 3)
    rows = 64 * 37                                                             # not a power of two
    grad, loss = sdd.sdd_mlp_grad(ctx, theta, norm, feats, targets, rows)
    Z = mlp.normalise(F[:rows], nv[:5], nv[5:])
    Y = Yall[:rows]
    th = _split(theta)
    g = grad.cpu().numpy().astype(np.float64)
    for f in range(2):
        L, want = mlp.loss_and_grad(th[f], Z, Y[:, f])
        got = g[f * STRIDE:f * STRIDE + P]
        err = np.abs(got - want)
        assert err.max() <= 2e-4 * np.abs(want).max(), (f, err.max(), np.abs(want).max())
        assert np.linalg.norm(got - want) <= 1e-4 * np.linalg.norm(want)
        assert abs(loss.cpu().numpy()[f] - L) <= 1e-5 * L


def test_adam_updates_match_oracle(sdd, mlp, oracle_mod):
    Pr, ctx = _front(oracle_mod, sdd)
    feats, targets, F, Y = _oracle_rows(mlp, Pr, 512, 4)                       # 5120 rows
    norm, nv = _oracle_norm(mlp, F)
    theta = _random_model(sdd, ctx, mlp, 5, scale=0.1)
    th0 = _split(theta)
    lr, steps = 1e-3, 4
    losses = sdd.sdd_mlp_train(ctx, theta, norm, feats, targets, epochs=3, batch=1024, lr=lr, max_steps=steps)
    Z = mlp.normalise(F, nv[:5], nv[5:])
    got = _split(theta)
    for f in range(2):
        want, wl = mlp.train(th0[f], Z, Y[:, f], epochs=3, batch=1024, lr0=lr, steps=steps)
        # the first loss is FP32 rounding only; later ones also carry the earlier updates' differences
        np.testing.assert_allclose(losses.cpu().numpy()[f][0], wl[0], rtol=1e-5)
        np.testing.assert_allclose(losses.cpu().numpy()[f], wl, rtol=1e-4)
        d = np.abs(got[f] - want)
        moved = np.abs(want - th0[f]).max()
        assert moved > 0.5 * lr
        # Adam moves every weight by about lr per step whatever the gradient's size, so a
        # gradient component lost in FP32 rounding can flip a step: allow that on a few
        assert np.mean(d <= 0.02 * lr * steps) >= 0.995, np.mean(d <= 0.02 * lr * steps)
        assert d.max() <= 2 * lr * steps + 1e-7


def _forward_mode_bound(mlp, th, mu, s, nf, tf):
    """FP64 table entries of one network at one slice, and a bound on the error of
    BF16 operands (relative 2^-8 per product) plus the approximate tanh."""
    ny, nx = nf["w"].shape
    X, Yg = np.meshgrid(np.arange(nx) / (nx - 1), np.arange(ny) / (ny - 1))
    n = nx * ny
    F = np.stack([X.ravel(), Yg.ravel(), np.full(n, tf), nf["w"].ravel(), nf["r"].ravel()], axis=1)
    Z = mlp.normalise(F, mu, s)
    p = mlp.unpack(th)
    h1 = np.tanh(Z @ p["W1"].T + p["b1"])
    k1 = 1 - h1 * h1
    out = []
    for comp in (0, 1):
        dF = np.zeros((n, 5))
        dF[:, comp] = 1.0
        dF[:, 3] = (nf["wx"] if comp == 0 else nf["wy"]).ravel()
        dF[:, 4] = (nf["rx"] if comp == 0 else nf["ry"]).ravel()
        u1 = k1 * ((dF * s) @ p["W1"].T)
        a2 = h1 @ p["W2"].T + p["b2"]
        h2 = np.tanh(a2)
        Wu = u1 @ p["W2"].T
        G = ((1 - h2 * h2) * Wu) @ p["w3"]
        S1 = (np.abs(1 - h2 * h2) * (np.abs(u1) @ np.abs(p["W2"]).T)) @ np.abs(p["w3"])
        S2 = (np.abs(Wu) * (np.abs(h1) @ np.abs(p["W2"]).T)) @ np.abs(p["w3"])
        out.append((G.reshape(ny, nx), (S1 + S2).reshape(ny, nx)))
    return out


def test_tensor_core_table_matches_forward_mode(sdd, mlp, oracle_mod):
    Pr, ctx = _front(oracle_mod, sdd, 69)        # 69 x 69 nodes: a ragged last tile of 16
    theta = _random_model(sdd, ctx, mlp, 9, scale=0.2)
    _, _, F, _ = _oracle_rows(mlp, Pr, 300, 9)
    norm, nv = _oracle_norm(mlp, F)
    K, S = 10, 3
    sdd.sdd_cv_tabulate(ctx, theta, norm, S, dt=1e-3, Dt=1e-2)
    T = sdd.sdd_cv_get_table(ctx, S).cpu().numpy()
    mu, s = nv[:5], nv[5:]
    th = _split(theta)
    # the oracle's table is the plain FP64 forward mode on the same node features
    want = mlp.tabulate(th, mu, s, Pr.w, K, S)
    nf = mlp.node_features(Pr.w)
    rel = []
    for q, tf in enumerate(mlp.slice_time_fracs(K, S)):
        for f in range(2):
            for comp, (G, B) in enumerate(_forward_mode_bound(mlp, th[f], mu, s, nf, tf)):
                np.testing.assert_allclose(want[q, ..., 2 * f + comp], G, rtol=1e-12, atol=1e-12)
                err = np.abs(T[q, ..., 2 * f + comp] - G)
                # BF16 operands (2^-8 per product), approximate tanh (< 2^-10); factor 2 margin
                assert np.all(err <= 2 * 2.0 ** -8 * B + 1e-6), (q, f, comp, (err / (B + 1e-30)).max())
                rel.append(np.sqrt(np.mean(err ** 2) / np.mean(G ** 2)))
    assert max(rel) < 0.02, rel


def test_trained_model_cuts_the_variance_and_keeps_the_mean(sdd, oracle_mod):
    P_, ctx = _heat(oracle_mod, sdd)
    dt, Dt = 1e-3, 0.05
    info = sdd.sdd_cv_train(ctx, per_horizon=4000, dt=dt, Dt=Dt, seed=1, epochs=5, batch=4096, lr=3e-3, init_seed=7)
    assert info["rows"] == 200000 and info["steps"] == 5 * (200000 // 4096) and info["slices"] == 50
    losses = sdd.sdd_cv_losses(ctx, info["steps"]).cpu().numpy()
    assert np.all(losses[:, -20:].mean(axis=1) < 0.8 * losses[:, 0])
    xs, ys = W.heat65_nodes()
    kw = dict(dt=dt, Dt=Dt, seed=0)
    plain = {k: v.cpu().numpy() for k, v in sdd.sdd_interface_mc(ctx, xs, ys, np.full(33, 2000), **kw).items()}
    sdd.sdd_cv_enable(ctx, True)
    cv = {k: v.cpu().numpy() for k, v in sdd.sdd_interface_mc(ctx, xs, ys, np.full(33, 2000), **kw).items()}
    inner = slice(1, 32)
    for f in ("xi", "eta"):
        ratio = (plain["se_" + f][inner] / cv["se_" + f][inner]) ** 2
        assert np.median(ratio) > 3, (f, np.median(ratio))
        d = np.abs(cv["mean_" + f] - plain["mean_" + f])[inner]
        assert np.all(d < 4 * np.hypot(cv["se_" + f], plain["se_" + f])[inner])


def test_learned_control_variate_meets_the_plain_error_with_fewer_path_steps(sdd, oracle_mod):
    """The w = 1 heat problem on 65 x 65 (33 nodes on x = 1/2, dt = 1e-3, Dt = 0.05):
    a network trained by the GPU on 1e6 single-path samples of the method, used as
    control variate with 2e3 paths per node, reaches the RMS error of the plain
    estimator with 1e4 paths per node, both against the FP64 oracle's estimate
    with 1e6 paths per node (whose own variance is taken out of both mean squared
    errors); and the plain estimator needs at least 4x the control variate's
    path-steps to reach the control variate's error (error^2 falls like 1/N)."""
    P_, ctx = _heat(oracle_mod, sdd)
    dt, Dt = 1e-3, 0.05
    info = sdd.sdd_cv_train(ctx, per_horizon=20000, dt=dt, Dt=Dt, seed=1, epochs=20, batch=4096, lr=3e-3,
                            init_seed=7)
    assert info["rows"] == 10 ** 6
    xs, ys = W.heat65_nodes()
    inner = np.arange(1, 32)
    xs, ys = xs[inner], ys[inner]

    def run(n, seed, cv):
        sdd.sdd_cv_enable(ctx, cv)
        o = sdd.sdd_interface_mc(ctx, xs, ys, np.full(xs.size, n), dt=dt, Dt=Dt, seed=seed)
        return {k: v.cpu().numpy() for k, v in o.items()}

    # the reference: the oracle's plain estimator at 1e6 paths per node (another seed)
    ref = oracle_mod.interface_mc(P_, xs, ys, 10 ** 6, dt=dt, Dt=Dt, seed=1000)
    ref_var = float(np.mean(np.concatenate([ref["se_xi"], ref["se_eta"]]) ** 2))
    reps = 12
    err_plain, err_cv, steps_plain, steps_cv = [], [], 0, 0
    for r in range(reps):
        a = run(10000, 2000 + r, False)
        b = run(2000, 3000 + r, True)
        err_plain.append(np.concatenate([a["mean_xi"] - ref["mean_xi"], a["mean_eta"] - ref["mean_eta"]]))
        err_cv.append(np.concatenate([b["mean_xi"] - ref["mean_xi"], b["mean_eta"] - ref["mean_eta"]]))
        steps_plain += a["path_steps"].sum()
        steps_cv += b["path_steps"].sum()
    mse_plain = float(np.mean(np.square(err_plain))) - ref_var
    mse_cv = float(np.mean(np.square(err_cv))) - ref_var
    assert mse_plain > 0 and mse_cv > 0, (mse_plain, mse_cv, ref_var)
    assert mse_cv <= mse_plain, (math.sqrt(mse_cv), math.sqrt(mse_plain))
    # plain path-steps needed for the control variate's error, against the control variate's
    assert steps_plain * (mse_plain / mse_cv) >= 4 * steps_cv, (steps_plain, steps_cv, mse_plain, mse_cv)
