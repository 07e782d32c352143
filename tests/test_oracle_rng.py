"""Pins of the oracle's variates: Philox4x32-10 and Box--Muller.

Philox is pinned against an independent implementation (triton's Philox in
interpreter mode on the CPU); Box--Muller against hand-derived special values
and the normal law.
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import stats

HERE = os.path.dirname(os.path.abspath(__file__))


def test_philox_matches_independent_implementation(oracle_mod):
    pytest.importorskip("triton")
    rng = np.random.default_rng(1234)
    req = []
    cases = []
    for seed in (0, 1, 0xDEADBEEF, 0x0123456789ABCDEF, 2 ** 64 - 1):
        ctrs = rng.integers(0, 2 ** 32, size=(16, 4), dtype=np.uint64).astype(np.uint32)
        ctrs[0] = 0
        ctrs[1] = [0xFFFFFFFF] * 4
        req.append([int(seed), ctrs.astype(np.int64).tolist()])
        cases.append((seed, ctrs))
    proc = subprocess.run([sys.executable, os.path.join(HERE, "_triton_philox_ref.py")],
                          input=json.dumps(req), capture_output=True, text=True, timeout=600)
    assert proc.returncode == 0, proc.stderr[-2000:]
    ref = json.loads(proc.stdout)
    for (seed, ctrs), want in zip(cases, ref):
        words, _ = oracle_mod.draw(seed, ctrs)
        np.testing.assert_array_equal(words.astype(np.int64), np.array(want, dtype=np.int64))


def test_counter_words_select_independent_streams(oracle_mod):
    # changing any one counter word (path, node, draw, step) changes the whole block
    base = np.array([[5, 9, 2, 7]], np.uint32)
    w0, _ = oracle_mod.draw(0x1111222233334444, base)
    for k in range(4):
        alt = base.copy()
        alt[0, k] += 1
        w1, _ = oracle_mod.draw(0x1111222233334444, alt)
        assert np.all(w0 != w1)


def test_philox_avalanche(oracle_mod):
    # flipping one counter bit flips about half of the 128 output bits
    rng = np.random.default_rng(7)
    base = rng.integers(0, 2 ** 32, size=(200, 4), dtype=np.uint64).astype(np.uint32)
    w0, _ = oracle_mod.draw(99, base)
    flips = []
    for word in range(4):
        for bit in (0, 13, 31):
            alt = base.copy()
            alt[:, word] ^= np.uint32(1 << bit)
            w1, _ = oracle_mod.draw(99, alt)
            x = np.bitwise_xor(w0, w1)
            flips.append(np.unpackbits(x.view(np.uint8)).sum() / x.shape[0])
    flips = np.array(flips)
    assert np.all(np.abs(flips - 64.0) < 4.0), flips


def test_philox_words_uniform(oracle_mod):
    ctr = np.zeros((50000, 4), np.uint32)
    ctr[:, 0] = np.arange(50000)
    ctr[:, 3] = 17
    w, _ = oracle_mod.draw(2024, ctr)
    for q in range(4):
        counts = np.bincount((w[:, q] >> 24).astype(np.int64), minlength=256)
        chi2 = ((counts - counts.mean()) ** 2 / counts.mean()).sum()
        assert stats.chi2.sf(chi2, 255) > 1e-4


def _word(m):
    """A 32-bit word whose low 23 bits are m (high bits arbitrary)."""
    return (0xA5 << 24) | m


def test_box_muller_special_values(oracle_mod):
    half = 1 << 22                    # u1 = (2^23 - 2^22) / 2^23 = 1/2
    R = math.sqrt(-2.0 * math.log(0.5))
    z0, z1 = oracle_mod.box_muller(_word(half), _word(0))             # angle 0
    assert z0 == pytest.approx(R, abs=1e-15) and z1 == pytest.approx(0.0, abs=1e-15)
    z0, z1 = oracle_mod.box_muller(_word(half), _word(1 << 21))       # angle pi/2
    assert z0 == pytest.approx(0.0, abs=1e-15) and z1 == pytest.approx(R, abs=1e-15)
    z0, z1 = oracle_mod.box_muller(_word(half), _word(1 << 22))       # angle pi
    assert z0 == pytest.approx(-R, abs=1e-15) and z1 == pytest.approx(0.0, abs=1e-15)
    z0, z1 = oracle_mod.box_muller(_word(0), _word(12345))            # u1 = 1: radius 0
    assert z0 == 0.0 and z1 == 0.0
    z0, z1 = oracle_mod.box_muller(_word((1 << 23) - 1), _word(0))    # smallest u1 = 2^-23
    assert z0 == pytest.approx(math.sqrt(2 * 23 * math.log(2)), rel=1e-14)


def test_normals_are_standard_normal(oracle_mod):
    n = 200000
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n) % 1000
    ctr[:, 1] = np.arange(n) // 1000
    _, z = oracle_mod.draw(0, ctr)
    flat = z.ravel()
    assert abs(flat.mean()) < 4 / math.sqrt(flat.size)
    assert abs(flat.var() - 1.0) < 4 * math.sqrt(2 / flat.size)
    assert stats.kstest(flat, "norm").pvalue > 1e-3
    # the two members of a pair are uncorrelated
    r = np.corrcoef(z[:, 0], z[:, 1])[0, 1]
    assert abs(r) < 4 / math.sqrt(n)
    # squared radius of a pair is exponential with mean 2
    r2 = z[:, 0] ** 2 + z[:, 1] ** 2
    assert stats.kstest(r2, "expon", args=(0, 2)).pvalue > 1e-3
