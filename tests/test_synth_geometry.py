"""Synthetic macro geometries: the random porous medium stand-in (Sec. 6.3)
has the stated porosity, non-overlapping periodic obstacles, fluid particles
outside every obstacle and wall particles within h of a surface."""
import numpy as np

from paper_2512_13267_gb300 import synth as S


def test_random_porous_medium_geometry():
    pos, is_wall, Lx, Ly, dh, c, r = S.random_porous_medium(seed=7)
    assert (Lx, Ly) == (12.0, 4.0) and len(r) == 17
    assert abs(1.0 - np.pi * np.sum(r ** 2) / (Lx * Ly) - 0.792) < 1e-12
    assert abs(r.mean() - 0.425) < 0.05
    box = np.array([Lx, Ly])
    for i in range(17):
        for j in range(i + 1, 17):
            d = c[i] - c[j]
            d -= box * np.rint(d / box)
            assert np.hypot(*d) >= r[i] + r[j] + 2 * dh - 1e-12
    depth = np.full(len(pos), -np.inf)
    for cc, R in zip(c, r):
        d = pos - cc
        d -= box * np.rint(d / box)
        depth = np.maximum(depth, R - np.hypot(d[:, 0], d[:, 1]))
    fluid = is_wall == 0
    assert np.all(depth[fluid] <= 0.0)
    assert np.all((depth[~fluid] > 0.0) & (depth[~fluid] <= 4 * dh + 1e-12))
    # walls come last; the lattice fluid fraction is close to the porosity
    assert np.all(np.diff(is_wall) >= 0)
    assert abs(fluid.sum() / ((Lx / dh) * (Ly / dh)) - 0.792) < 0.01
