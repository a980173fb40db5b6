"""Pins of the oracle's Philox4x32-10 and of the per-cell draws built on it."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert list(orc.philox(ctr, key)) == want


def test_cell_draws_use_lanes_0_and_1(orc):
    # counter (cell, run, step, fire), key (seed lo, seed hi); u = (x >> 8) * 2^-24
    seed = 0x0123456789ABCDEF
    x = orc.philox([77, 3, 11, 5], [seed & 0xFFFFFFFF, seed >> 32])
    u0, u1 = orc.cell_draws(seed, 3, 11, 5, 77)
    assert u0 == (int(x[0]) >> 8) / 2.0 ** 24
    assert u1 == (int(x[1]) >> 8) / 2.0 ** 24


def test_uniform_draws_moments(orc):
    # 20000 counters: mean 1/2 and variance 1/12 within 5 standard errors, and the two
    # lanes uncorrelated; a wrong shift or a reused lane fails this.
    u0 = np.empty(20000)
    u1 = np.empty(20000)
    for k in range(20000):
        u0[k], u1[k] = orc.cell_draws(7, k % 13, k // 13, 0, k * 7919)
    n = len(u0)
    for u in (u0, u1):
        assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
        assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / n)
        assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(np.corrcoef(u0, u1)[0, 1]) < 5 / np.sqrt(n)
