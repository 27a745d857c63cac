"""Pins of the oracle's counter-based random stream (reading R3).

The random force needs theta_ij = theta_ji ~ N(0,1), reproducible from
(box, pair, step).  The generator is Philox4x32-10; its known-answer vectors
are published with the method, and the Box-Muller map is checked against the
normal distribution."""
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat_rows())
def test_philox_known_answers(ctr, key, out):
    assert O.philox4x32_10(ctr, key) == out


def test_theta_symmetric_and_keyed():
    for (i, j) in [(0, 1), (5, 4000), (77, 3)]:
        a = O.pair_theta(1, 3, i, j, 17)
        b = O.pair_theta(1, 3, j, i, 17)
        assert a == b
    # a different step, box or seed gives a different draw
    base = O.pair_theta(1, 3, 5, 9, 17)
    assert O.pair_theta(1, 3, 5, 9, 18) != base
    assert O.pair_theta(1, 4, 5, 9, 17) != base
    assert O.pair_theta(2, 3, 5, 9, 17) != base


def test_consecutive_seeds_do_not_share_a_box_stream():
    # R3 keys by (seed_lo, seed_hi ^ box): (seed s, box b) and (s ^ 1, b ^ 1)
    # must draw different noise (a key of seed_lo ^ box would make them equal)
    for s in (0, 1, 2, 7, 1000):
        for b in (0, 1, 5, 1023):
            for (i, j, step) in [(0, 1, 1), (17, 230, 99)]:
                assert O.pair_theta(s, b, i, j, step) != O.pair_theta(s ^ 1, b ^ 1, i, j, step)
    # the documented key and counter layout, through the raw generator
    seed, box, i, j, step = (5 << 32) | 123, 77, 900, 14, (3 << 32) | 41
    w = O.philox4x32_10([j, i, step & 0xFFFFFFFF, step >> 32],
                        [seed & 0xFFFFFFFF, (seed >> 32) ^ box])
    assert O.pair_theta(seed, box, i, j, step) == O.theta_from_words(w[0], w[1])


def test_theta_is_standard_normal():
    th = np.array([O.pair_theta(11, 0, i, i + 1 + (i % 7), 3) for i in range(20000)])
    assert abs(th.mean()) < 4 / np.sqrt(th.size)
    assert abs(th.var() - 1.0) < 4 * np.sqrt(2.0 / th.size)
    assert stats.kstest(th, "norm").pvalue > 1e-3


def test_box_muller_grid_extremes():
    # u1, u2 live on the 2^-23 grid offset by half a cell: the smallest u1 gives
    # the largest |theta| = sqrt(2 * 24 ln 2) and never log(0)
    top = O.theta_from_words(0x000001FF, 0x00000000)
    assert np.isclose(top, np.sqrt(-2 * np.log(0.5 / 2**23)) * np.cos(2 * np.pi * 0.5 / 2**23),
                      rtol=1e-14)
    # the low 9 bits are dropped
    assert O.theta_from_words(0x12345600, 0xABCDEE00) == O.theta_from_words(0x123457FF, 0xABCDEFFF)
    # u1 = 1/2, u2 = 1/4 + half cell: theta = sqrt(2 ln 2) cos(pi/2 + eps) ~ 0
    assert abs(O.theta_from_words(0x80000000, 0x40000000)) < 1e-6
