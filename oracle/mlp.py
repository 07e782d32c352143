"""FP64 reference of the learned control variate (test infrastructure).

TEST INFRASTRUCTURE ONLY: called by the test suite, the smoke check and the
benchmark's CPU legs; the product library never uses it.

The paper estimates the interface values by plain Monte Carlo means (Sec. 4)
and notes that their convergence is slow. The control variate subtracts, path
by path, the sum of G(s_j, X_j) . sqrt(2) dW_j over the sub-steps the path
takes, with G a model of the gradient of the solution of Eq. (6) in space; any
G leaves the mean unchanged (a martingale stopped at a bounded time). Here G is
the spatial gradient of a small network g(x, y, t, w, |grad w|/w) fitted to the
method's own single-path scores:

  features f = (x, y, t / Dt, w(x, y), r(x, y)), r = |grad w| / w, w and r
             interpolated bilinearly from their node values; t the time left
             in the mesh step (Eq. 7b runs backward in time);
  z = (f - mu) * s, the standardisation fitted on the training set (s = 1 /
             standard deviation, 0 for a feature that does not vary);
  g(z) = w3 . tanh(W2 tanh(W1 z + b1) + b2) + b3, widths 5 -> 64 -> 64 -> 1,
             one network for xi and one for eta;
  loss      mean squared error against the single-path scores Y (their
             conditional mean given the start is the solution, so the
             regression target is unbiased);
  Adam (Kingma & Ba 2015, Algorithm 1) with a cosine learning-rate decay.

The table G the estimator reads is the total derivative of g in x and y at
every node, taken by forward-mode differentiation through the features
(d/dx of w and r by the finite differences of the drift, Sec. 4), at one time
per slice of sub-steps.

Parameter vector of one network (float64 here, float32 on the device), in
this order: W1 (64 x 5, row-major, [out][in]), b1 (64), W2 (64 x 64,
[out][in]), b2 (64), w3 (64), b3 (1): 4609 values.

Every function here is the plain definition; nothing is blocked or fused.
"""
from __future__ import annotations

import math

import numpy as np

D = 5            # inputs
H = 64           # hidden width
P = H * D + H + H * H + H + H + 1   # 4609 parameters per network

_OFF = {}
_o = 0
for _name, _size in (("W1", H * D), ("b1", H), ("W2", H * H), ("b2", H), ("w3", H), ("b3", 1)):
    _OFF[_name] = (_o, _o + _size)
    _o += _size
assert _o == P

INIT_WORD = 0x494E4954   # counter word of the initial weights ("INIT")
SAMPLE_STEP_WORD = 0xFFFFFFFF  # step word of the training paths' Philox counters


def unpack(theta):
    """Views of one network's parameters: W1 (H, D), b1, W2 (H, H), b2, w3, b3 (scalar array)."""
    t = np.asarray(theta)
    assert t.shape == (P,)

    def v(name, shape):
        a, b = _OFF[name]
        return t[a:b].reshape(shape)
    return dict(W1=v("W1", (H, D)), b1=v("b1", (H,)), W2=v("W2", (H, H)), b2=v("b2", (H,)),
                w3=v("w3", (H,)), b3=v("b3", (1,)))


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2), np.ravel(b2), np.ravel(w3),
                           np.ravel(b3)]).astype(np.float64)


def _philox_words(seed: int, counters):
    from . import draw
    words, _ = draw(seed, counters)
    return words


def init_params(seed: int):
    """Initial weights of the two networks, shape (2, P).

    Glorot-uniform weights (limit sqrt(6 / (fan_in + fan_out))), zero biases.
    The uniform of weight p of network f comes from word 0 of the Philox4x32-10
    block with key seed and counter (p, f, INIT_WORD, 0):
    u = ((word >> 8) + 0.5) 2^-24, weight = (2u - 1) limit, rounded to FP32."""
    out = np.zeros((2, P))
    for f in range(2):
        ctr = np.zeros((P, 4), np.uint32)
        ctr[:, 0] = np.arange(P, dtype=np.uint32)
        ctr[:, 1] = f
        ctr[:, 2] = INIT_WORD
        words = _philox_words(seed, ctr)[:, 0].astype(np.float64)
        u = (np.floor(words / 256.0) + 0.5) * 2.0 ** -24
        theta = np.zeros(P)
        for name, fan_in, fan_out in (("W1", D, H), ("W2", H, H), ("w3", H, 1)):
            a, b = _OFF[name]
            limit = math.sqrt(6.0 / (fan_in + fan_out))
            theta[a:b] = (2.0 * u[a:b] - 1.0) * limit
        out[f] = theta.astype(np.float32).astype(np.float64)
    return out


# ---------------------------------------------------------------- features

def fd_grad(f):
    """d/dx, d/dy of node values on the unit square by the finite differences
    of the drift (Sec. 4): central in the interior, second-order one-sided
    (-3 f0 + 4 f1 - f2) / 2h on the edges. f[j, i] at x = i h_x, y = j h_y."""
    f = np.asarray(f, dtype=np.float64)
    ny, nx = f.shape
    hx, hy = 1.0 / (nx - 1), 1.0 / (ny - 1)
    gx = np.zeros_like(f)
    gy = np.zeros_like(f)
    gx[:, 1:-1] = (f[:, 2:] - f[:, :-2]) / (2 * hx)
    gx[:, 0] = (-3 * f[:, 0] + 4 * f[:, 1] - f[:, 2]) / (2 * hx)
    gx[:, -1] = (3 * f[:, -1] - 4 * f[:, -2] + f[:, -3]) / (2 * hx)
    gy[1:-1, :] = (f[2:, :] - f[:-2, :]) / (2 * hy)
    gy[0, :] = (-3 * f[0, :] + 4 * f[1, :] - f[2, :]) / (2 * hy)
    gy[-1, :] = (3 * f[-1, :] - 4 * f[-2, :] + f[-3, :]) / (2 * hy)
    return gx, gy


def node_features(w):
    """Node fields the network reads: w, r = |grad w| / w and their gradients."""
    w = np.asarray(w, dtype=np.float64)
    wx, wy = fd_grad(w)
    r = np.sqrt(wx * wx + wy * wy) / w
    rx, ry = fd_grad(r)
    return dict(w=w, r=r, wx=wx, wy=wy, rx=rx, ry=ry)


def _bilinear_many(f, xs, ys):
    """Bilinear interpolation of node values at many points (Sec. 4)."""
    ny, nx = f.shape
    u = np.clip(np.asarray(xs) * (nx - 1), 0.0, nx - 1.0)
    v = np.clip(np.asarray(ys) * (ny - 1), 0.0, ny - 1.0)
    i = np.minimum(np.floor(u).astype(np.int64), nx - 2)
    j = np.minimum(np.floor(v).astype(np.int64), ny - 2)
    s, t = u - i, v - j
    return ((1 - s) * (1 - t) * f[j, i] + s * (1 - t) * f[j, i + 1] + (1 - s) * t * f[j + 1, i]
            + s * t * f[j + 1, i + 1])


def features(nf, xs, ys, t_frac):
    """Raw features (n, 5) at points (xs, ys) with time left t_frac * Dt."""
    xs = np.asarray(xs, dtype=np.float64)
    n = xs.shape[0]
    F = np.zeros((n, D))
    F[:, 0] = xs
    F[:, 1] = ys
    F[:, 2] = t_frac
    F[:, 3] = _bilinear_many(nf["w"], xs, ys)
    F[:, 4] = _bilinear_many(nf["r"], xs, ys)
    return F


def standardise(F):
    """(mu, s): mean and inverse population standard deviation of each feature;
    s = 0 where the standard deviation is below 1e-6 max(1, |mu|)."""
    F = np.asarray(F, dtype=np.float64)
    mu = F.mean(axis=0)
    sd = np.sqrt(((F - mu) ** 2).mean(axis=0))
    s = np.where(sd > 1e-6 * np.maximum(1.0, np.abs(mu)), 1.0 / np.where(sd > 0, sd, 1.0), 0.0)
    return mu, s


def normalise(F, mu, s):
    return (np.asarray(F, dtype=np.float64) - mu) * s


# ---------------------------------------------------------------- network

def forward(theta, Z):
    """g(z) for the rows of Z (n, 5); returns (out (n,), cache)."""
    p = unpack(theta)
    a1 = Z @ p["W1"].T + p["b1"]
    h1 = np.tanh(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(a2)
    out = h2 @ p["w3"] + p["b3"][0]
    return out, (Z, h1, h2)


def loss_and_grad(theta, Z, Y):
    """Mean squared error over the rows and its gradient by backpropagation."""
    p = unpack(theta)
    out, (Z, h1, h2) = forward(theta, Z)
    n = Z.shape[0]
    e = out - np.asarray(Y, dtype=np.float64)
    L = float(np.mean(e * e))
    d = 2.0 * e / n                          # dL/d out
    gw3 = h2.T @ d
    gb3 = np.array([d.sum()])
    g2 = np.outer(d, p["w3"]) * (1.0 - h2 * h2)   # dL/d a2
    gW2 = g2.T @ h1
    gb2 = g2.sum(axis=0)
    g1 = (g2 @ p["W2"]) * (1.0 - h1 * h1)         # dL/d a1
    gW1 = g1.T @ Z
    gb1 = g1.sum(axis=0)
    return L, pack(gW1, gb1, gW2, gb2, gw3, gb3)


def input_grad(theta, Z, dZx, dZy):
    """g and its derivatives along the input directions dZx, dZy (forward mode)."""
    p = unpack(theta)
    a1 = Z @ p["W1"].T + p["b1"]
    h1 = np.tanh(a1)
    k1 = 1.0 - h1 * h1
    u1 = k1 * (dZx @ p["W1"].T)
    v1 = k1 * (dZy @ p["W1"].T)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(a2)
    k2 = 1.0 - h2 * h2
    u2 = k2 * (u1 @ p["W2"].T)
    v2 = k2 * (v1 @ p["W2"].T)
    return h2 @ p["w3"] + p["b3"][0], u2 @ p["w3"], v2 @ p["w3"]


def adam_update(theta, m, v, g, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """Step t (counting from 1) of Adam (Kingma & Ba 2015, Algorithm 1)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def lr_at(step: int, total: int, lr0: float) -> float:
    """Cosine decay from lr0 (step 0) towards 0 (step total)."""
    return lr0 * 0.5 * (1.0 + math.cos(math.pi * step / total))


def train(theta0, Z, Y, *, epochs: int, batch: int, lr0: float, steps=None):
    """Minibatch Adam on the rows in their stored order: epoch after epoch, batch b
    takes rows [b batch, (b + 1) batch); a trailing partial batch is dropped.
    steps, if given, stops after that many updates. Returns (theta, losses)."""
    theta = np.array(theta0, dtype=np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    nb = Z.shape[0] // batch
    total = epochs * nb
    losses = []
    t = 0
    for e in range(epochs):
        for b in range(nb):
            if steps is not None and t >= steps:
                return theta, losses
            rows = slice(b * batch, (b + 1) * batch)
            L, g = loss_and_grad(theta, Z[rows], Y[rows])
            losses.append(L)
            theta, m, v = adam_update(theta, m, v, g, t + 1, lr_at(t, total, lr0))
            t += 1
    return theta, losses


# ---------------------------------------------------------------- the table

def slice_bounds(K: int, S: int):
    """First sub-step of each slice: slice q serves the j with floor(j S / K) = q."""
    return [(q * K + S - 1) // S for q in range(S + 1)]


def slice_time_fracs(K: int, S: int):
    """Time left, as a fraction of Dt, at the middle of each slice's sub-steps."""
    b = slice_bounds(K, S)
    return [(K - 0.5 * (b[q] + b[q + 1] - 1)) / K for q in range(S)]


def tabulate(thetas, mu, s, w, K: int, S: int):
    """The control-variate table (S, ny, nx, 4): d/dx, d/dy of the xi network,
    then of the eta network, at every node, at the time of each slice."""
    nf = node_features(w)
    ny, nx = nf["w"].shape
    X, Yg = np.meshgrid(np.arange(nx) / (nx - 1), np.arange(ny) / (ny - 1))
    n = nx * ny
    dFx = np.zeros((n, D))
    dFy = np.zeros((n, D))
    dFx[:, 0] = 1.0
    dFy[:, 1] = 1.0
    dFx[:, 3] = nf["wx"].ravel()
    dFy[:, 3] = nf["wy"].ravel()
    dFx[:, 4] = nf["rx"].ravel()
    dFy[:, 4] = nf["ry"].ravel()
    T = np.zeros((S, ny, nx, 4))
    for q, tf in enumerate(slice_time_fracs(K, S)):
        F = np.stack([X.ravel(), Yg.ravel(), np.full(n, tf), nf["w"].ravel(), nf["r"].ravel()], axis=1)
        Z = normalise(F, mu, s)
        for f in range(2):
            _, gx, gy = input_grad(thetas[f], Z, dFx * s, dFy * s)
            T[q, ..., 2 * f] = gx.reshape(ny, nx)
            T[q, ..., 2 * f + 1] = gy.reshape(ny, nx)
    return T


def field_gradient_table(xi, eta):
    """The control variate without training: one slice holding the finite-
    difference gradients of the fields at t_{n-1} (Sec. 4's differences). Over
    a short mesh step the solution's gradient stays close to it."""
    gx, gy = fd_grad(xi)
    hx, hy = fd_grad(eta)
    return np.stack([gx, gy, hx, hy], axis=-1)[None]


CV_CELL_ORDER = 33


def binomial_weights(order: int):
    """C(order, m) 2^-order, m = 0..order: the binomial smoothing filter."""
    return np.array([math.comb(order, m) for m in range(order + 1)], dtype=np.float64) / 2.0 ** order


def field_cell_gradient_table(xi, eta, order: int = CV_CELL_ORDER):
    """The untrained control variate as one value per cell: the finite-difference
    gradients of the fields at t_{n-1} (field_gradient_table) smoothed by the
    binomial filter of odd order `order` along x, then along y, centred on the
    cells: cell i takes node i - r + m with weight C(order, m) 2^-order,
    m = 0..order, r = (order - 1) / 2, nodes past an edge replaced by the edge
    node. The smoothing removes the grid-scale noise that the interface
    values' Monte Carlo error leaves in the fields' differences; any model keeps
    the estimate unbiased. Shape (1, ny - 1, nx - 1, 4)."""
    if order < 1 or order % 2 != 1:
        raise ValueError("the smoothing order must be odd and positive")
    g = field_gradient_table(xi, eta)[0]
    wts = binomial_weights(order)
    r = (order - 1) // 2
    for axis in (1, 0):
        L = g.shape[axis]
        out = np.zeros_like(np.take(g, np.arange(L - 1), axis=axis))
        for m, wm in enumerate(wts):
            out += wm * np.take(g, np.clip(np.arange(L - 1) - r + m, 0, L - 1), axis=axis)
        g = out
    return g[None]


# ---------------------------------------------------------------- training data

def sample_starts(seed: int, words):
    """Start points of the training paths: words 0, 1 of the Philox block with
    counter (1, word, 0, SAMPLE_STEP_WORD), each u = ((bits >> 8) + 0.5) 2^-24."""
    words = np.asarray(words, dtype=np.uint32)
    ctr = np.zeros((words.size, 4), np.uint32)
    ctr[:, 0] = 1
    ctr[:, 1] = words
    ctr[:, 3] = SAMPLE_STEP_WORD
    r = _philox_words(seed, ctr).astype(np.float64)
    return (np.floor(r[:, 0] / 256.0) + 0.5) * 2.0 ** -24, (np.floor(r[:, 1] / 256.0) + 0.5) * 2.0 ** -24


def training_samples(problem, *, per_horizon: int, dt: float, Dt: float, seed: int, exit_mode: int = 0,
                     threads=None):
    """The method's own samples: for every horizon k = 1..K sub-steps, per_horizon
    single paths from start points uniform in the unit square, each run k
    sub-steps of the estimator (node word (k - 1) per_horizon + m, step word
    SAMPLE_STEP_WORD). Row m K + (k - 1) holds sample m of horizon k.
    Returns (F (n, 5) raw features, Y (n, 2) scores)."""
    from . import interface_mc, sub_steps
    K = sub_steps(dt, Dt)
    M = per_horizon
    nf = node_features(problem.w)
    F = np.zeros((M * K, D))
    Y = np.zeros((M * K, 2))
    for k in range(1, K + 1):
        words = (np.arange(M, dtype=np.uint64) + (k - 1) * M).astype(np.uint32)
        xs, ys = sample_starts(seed, words)
        r = interface_mc(problem, xs, ys, 1, dt=dt, Dt=k * dt, seed=seed, exit_mode=exit_mode,
                         step_index=SAMPLE_STEP_WORD, node_ids=words, threads=threads)
        rows = np.arange(M) * K + (k - 1)
        F[rows] = features(nf, xs, ys, k / K)
        Y[rows, 0] = r["mean_xi"]
        Y[rows, 1] = r["mean_eta"]
    return F, Y
