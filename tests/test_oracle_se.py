"""Pins of the oracle's standard error (Sec. 4 replaces the expectations of
Eq. 7b by arithmetic means; reading R11: the N - 1 sample variance, SE = s/sqrt(N)).

Every statistical tolerance of the parity tests is a multiple of this SE, so
it is pinned from both sides: against the per-path scores the oracle itself
reports (numpy's ddof=1 standard deviation, an independent routine), and
against the spread of the node means over independent seeds, which an SE too
large or too small by any fixed factor (a dropped sqrt, an N for an N - 1 at
small N, a variance of the wrong field) would not match.
"""
import math

import numpy as np

import workloads as W


def _problem(oracle_mod, n=33):
    # a drift that varies over the domain, the Winslow face data, xi0 = x, eta0 = y
    w = W.w_front(n, 0.1).astype(np.float64)
    xi0, eta0 = W.identity_fields(n)
    return oracle_mod.Problem(w, xi0, eta0)


def test_se_is_the_sample_deviation_of_the_path_scores_over_sqrt_n(oracle_mod):
    P = _problem(oracle_mod)
    xs = np.array([0.5, 0.31, 0.07, 0.5, 0.9, 0.5])
    ys = np.array([0.5, 0.44, 0.5, 0.03, 0.2, 0.5])
    npaths = np.array([400, 1000, 77, 250, 2, 1])
    for mode in (0, 1, 2):
        r = oracle_mod.interface_mc(P, xs, ys, npaths, dt=5e-4, Dt=0.02, seed=3, exit_mode=mode, record=True)
        off = np.concatenate([[0], np.cumsum(npaths)])
        for k in range(xs.size):
            for f in ("xi", "eta"):
                v = r["score_" + f][off[k]:off[k + 1]]
                n = v.size
                want_se = np.std(v, ddof=1) / math.sqrt(n) if n > 1 else 0.0
                np.testing.assert_allclose(r["mean_" + f][k], np.mean(v), rtol=0, atol=1e-14)
                np.testing.assert_allclose(r["se_" + f][k], want_se, rtol=1e-12, atol=1e-16,
                                           err_msg=f"mode {mode} node {k} {f}")
        # node 4 has two paths: SE = |Y1 - Y2| / 2 exactly (s^2 = (Y1 - Y2)^2 / 2, N = 2)
        a, b = r["score_xi"][off[4]:off[4] + 2]
        np.testing.assert_allclose(r["se_xi"][4], abs(a - b) / 2, rtol=1e-12, atol=1e-16)
        # a single path has no spread estimate
        assert r["se_xi"][5] == 0.0 and r["se_eta"][5] == 0.0


def test_se_matches_the_spread_of_the_means_over_independent_seeds(oracle_mod):
    # M independent estimates of each node: the variance of the means around
    # their average, over the mean squared SE, is chi^2 / dof with
    # dof = nodes x (M - 1) (sampled at N = 200, where s^2 is close to sigma^2)
    P = _problem(oracle_mod)
    xs = np.array([0.5, 0.5, 0.25, 0.7, 0.12, 0.5])
    ys = np.array([0.5, 0.2, 0.5, 0.65, 0.3, 0.9])
    M, N = 40, 200
    means = {"xi": [], "eta": []}
    ses = {"xi": [], "eta": []}
    for s in range(M):
        r = oracle_mod.interface_mc(P, xs, ys, N, dt=1e-3, Dt=0.03, seed=1000 + s, step_index=s % 3)
        for f in means:
            means[f].append(r["mean_" + f])
            ses[f].append(r["se_" + f])
    dof = xs.size * (M - 1)
    # two-sided 99.9% bounds of chi^2_dof / dof by the Wilson-Hilferty approximation
    z = 3.29
    lo = (1 - 2 / (9 * dof) - z * math.sqrt(2 / (9 * dof))) ** 3
    hi = (1 - 2 / (9 * dof) + z * math.sqrt(2 / (9 * dof))) ** 3
    for f in means:
        m = np.array(means[f])       # (M, nodes)
        se = np.array(ses[f])
        spread = np.sum((m - m.mean(axis=0)) ** 2, axis=0) / (M - 1)   # per node
        ratio = float(np.sum(spread) / np.sum(np.mean(se ** 2, axis=0)))
        assert lo <= ratio <= hi, (f, ratio, lo, hi)
        # and the standardised deviations of single estimates are not all tiny
        zdev = (m - m.mean(axis=0)) / se
        assert 0.6 < float(np.std(zdev)) < 1.4, (f, float(np.std(zdev)))
