"""Comparison helpers for the CUDA path against the oracle (same Philox streams)."""
import numpy as np

# The estimator's own tolerance: per node within 3 standard errors; exit
# decisions identical for at least 99.9% of paths. Paths whose exit decision
# agrees carry single-precision rounding only: their scores and end points
# agree to well below 1e-4.
EXIT_AGREEMENT = 0.999
PATH_TOL = 1e-4
NODE_TOL = 1e-4


def compare_records(g, o):
    """g: GPU records (numpy), o: oracle records. Returns (agree mask, report dict)."""
    code_g = np.asarray(g["code"])
    code_o = np.asarray(o["code"])
    same = (code_g == code_o) & (np.asarray(g["steps"]) == np.asarray(o["steps"]))
    frac = same.mean() if same.size else 1.0
    rep = {"paths": int(same.size), "disagree": int((~same).sum()), "agree_frac": float(frac)}
    if same.any():
        for k in ("score_xi", "score_eta", "x_end", "y_end"):
            rep["max_" + k] = float(np.abs(np.asarray(g[k], np.float64)[same] - np.asarray(o[k])[same]).max())
    return same, rep


def assert_records(g, o, score_tol=PATH_TOL):
    same, rep = compare_records(g, o)
    assert rep["agree_frac"] >= EXIT_AGREEMENT, rep
    for k in ("score_xi", "score_eta", "x_end", "y_end"):
        if "max_" + k in rep:
            assert rep["max_" + k] <= (score_tol if k.startswith("score") else PATH_TOL), rep
    return same, rep


def assert_nodes(g, o, n_paths, same=None, offsets=None):
    """Per node: |mean_gpu - mean_oracle| <= 3 SE, and <= 1e-4 on every node whose
    paths all agree; SE, exit and step counts consistent."""
    clean_all = None
    if same is not None and offsets is not None:
        clean_all = np.array([same[offsets[k]:offsets[k + 1]].all() for k in range(len(offsets) - 1)])
    for f in ("xi", "eta"):
        d = np.abs(np.asarray(g["mean_" + f]) - np.asarray(o["mean_" + f]))
        se = np.asarray(o["se_" + f])
        # nodes whose paths all agree carry only rounding (<= 1e-4); the others <= 3 SE
        allow = 3 * se + (NODE_TOL * clean_all if clean_all is not None else 1e-12)
        assert np.all(d <= allow), (f, d.max(), np.argmax(d - allow))
        if same is not None and offsets is not None:
            clean = clean_all
            if clean.any():
                assert d[clean].max() <= NODE_TOL, (f, d[clean].max())
            gse = np.asarray(g["se_" + f])
            rel = np.abs(gse[clean] - se[clean]) / np.maximum(se[clean], 1e-12)
            if clean.any():
                assert np.all((rel <= 1e-3) | (se[clean] < 1e-9)), (f, rel.max())
    if same is not None and offsets is not None:
        clean = np.array([same[offsets[k]:offsets[k + 1]].all() for k in range(len(offsets) - 1)])
        np.testing.assert_array_equal(np.asarray(g["n_exit"])[clean], np.asarray(o["n_exit"])[clean])
        np.testing.assert_array_equal(np.asarray(g["path_steps"])[clean], np.asarray(o["path_steps"])[clean])


def assert_flips_near_boundary(oracle_mod, P, xs, ys, n_paths, g, o, same, *, dt, Dt, seed, step_index=0,
                               node_ids=None, tol=1e-4):
    """Paths whose exit decision differs (plain exit test): the oracle's path
    must have come within tol of a boundary line by the first sub-step where
    the two decisions can differ (the GPU decides in single precision, the
    oracle in double; away from the boundary both decide alike)."""
    flips = np.flatnonzero(~np.asarray(same))
    if flips.size == 0:
        return 0
    n_paths = np.broadcast_to(np.asarray(n_paths, np.int64), (len(xs),))
    offs = np.concatenate([[0], np.cumsum(n_paths)])
    node = np.searchsorted(offs, flips, side="right") - 1
    path = flips - offs[node]
    ids = np.arange(len(xs), dtype=np.uint32) if node_ids is None else np.asarray(node_ids, np.uint32)
    upto = np.minimum(np.asarray(g["steps"])[flips], np.asarray(o["steps"])[flips])
    m = oracle_mod.path_margins(P, np.asarray(xs)[node], np.asarray(ys)[node], ids[node], path, upto, dt=dt,
                                Dt=Dt, seed=seed, step_index=step_index)
    assert np.all(m <= tol), (flips[m > tol][:10], m[m > tol][:10])
    return flips.size


def assert_trajectory_step(g, o, gfields, ofields, prev_gap, slack=0.0, se=None, tag="", clean=True):
    """One mesh step of the GPU's trajectory against the oracle's own trajectory from the
    same seeded start (neither side ever reads the other's fields). The paths of both sides
    move alike (the drift comes from w) and a surviving path scores the previous fields,
    bilinearly, which differ by at most prev_gap: the node means may differ by 3 standard
    errors (exit decisions that flip) plus prev_gap, plus `slack`. The implicit subdomain
    solve maps the interface values and the previous fields to the new fields by a
    nonnegative matrix whose rows sum to 1 (an M-matrix system, R14): the new fields differ
    by at most the larger of the interface values' and the previous fields' gaps (plus the
    iterative solve's tolerance). se: the standard errors of the comparison (default the
    oracle's). clean: also require 90% of the nodes within rounding (1e-4) of the bound's
    deterministic part (not where the two sides' control-variate models differ by construction).
    Returns the new fields' gap."""
    iface = 0.0
    for f in ("xi", "eta"):
        d = np.abs(np.asarray(g["mean_" + f]) - np.asarray(o["mean_" + f]))
        s = np.asarray(o["se_" + f]) if se is None else np.asarray(se[f])
        assert np.all(d <= 3 * s + prev_gap + slack + 1e-12), (tag, f, d.max(), prev_gap)
        # most nodes move by rounding and the previous fields' gap only
        if clean:
            assert np.mean(d <= NODE_TOL + prev_gap + slack) >= 0.9, (tag, f, np.mean(d <= NODE_TOL + prev_gap + slack))
        iface = max(iface, float(d.max()))
    gap = max(float(np.abs(gfields[0] - ofields[0]).max()), float(np.abs(gfields[1] - ofields[1]).max()))
    assert gap <= max(iface, prev_gap) + 1e-9, (tag, gap, iface, prev_gap)
    return gap
