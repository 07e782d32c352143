"""The cluster multigrid kernel indexes its coarse levels with single-precision
quotients: floor(k / d) is taken as trunc((k + 1/2) * fl(1/d)) in float32 with
round-to-nearest products. That is exact while (k + 1/2) d < 2^22; the host
admits a level only if W^2 (my + 2) < 2^21, W = mx + 2, which bounds every (k, d)
the kernel forms (sweeps: d = (mx + 1) / 2, k < d my; restriction: d = W,
k < W (my + 2); prolongation: d = mx, k < mx my). Checked here exhaustively in
float32 over that whole range.
"""
import numpy as np

BOUND = 1 << 21


def _qdiv(k, d):
    rd = np.float32(1.0) / np.float32(d)                     # correctly rounded reciprocal
    prod = (k.astype(np.float32) + np.float32(0.5)) * rd     # one rounding
    return np.trunc(prod).astype(np.int64)


def test_float_quotient_is_exact_below_the_admitted_bound():
    checked = 0
    for d in range(1, 2049):
        kmax = BOUND // d + 1        # k d < 2^21 covers every k the admitted levels form with this d
        k = np.arange(kmax, dtype=np.int64)
        np.testing.assert_array_equal(_qdiv(k, d), k // d, err_msg=f"d={d}")
        checked += kmax
    assert checked > 10_000_000


def test_admitted_levels_stay_inside_the_checked_range():
    # every odd level shape with W^2 (my + 2) < 2^21 forms only (k, d) with k d < 2^21
    for mx in range(1, 2048, 2):
        W = mx + 2
        my_max = BOUND // (W * W) - 2
        for my in (1, 3, max(1, my_max - (1 - my_max % 2))):
            if my < 1 or W * W * (my + 2) >= BOUND:
                continue
            per_row = (mx + 1) // 2
            assert per_row * my * per_row < BOUND          # sweeps
            assert W * (my + 2) * W < BOUND                # restriction
            assert mx * my * mx < BOUND                    # prolongation


def test_the_quotient_fails_far_outside_the_bound():
    # the bound is not vacuous: for large enough k d the float product does round across an integer
    d = 3
    k = np.arange(1 << 24, (1 << 24) + 4096, dtype=np.int64)
    assert np.any(_qdiv(k, d) != k // d)
