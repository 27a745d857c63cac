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


def test_carreau_yasuda_fit_recovers_known_parameters():
    # data drawn from the paper's N_d = 8 curve (its CY table) at 8 rates,
    # 1 % noise: the fit recovers eta0 and the curve; lambda trades off
    # against n and eta_inf over two decades of rate, so only its scale is
    # fixed by such data
    from paper_2512_13267_gb300 import rheometry as R
    rng = np.random.default_rng(0)
    g = np.array([0.0005, 0.001, 0.002, 0.005, 0.01, 0.02, 0.05, 0.1])
    true = R.carreau_yasuda(g, 34.29, 3.15, 89.75, 0.95, 0.37)
    eta = true * (1 + 0.01 * rng.standard_normal(8))
    fit = R.fit_carreau_yasuda(g, eta, 0.01 * eta)
    assert abs(fit["eta0"] / 34.29 - 1) < 0.1, fit
    assert 0.5 < fit["lam"] / 89.75 < 2.0, fit
    assert fit["rms_log_residual"] < 0.03
    curve = R.carreau_yasuda(g, fit["eta0"], fit["eta_inf"], fit["lam"], fit["a"], fit["n"])
    assert np.all(np.abs(curve / true - 1) < 0.03)
    # a Newtonian plateau is a flat fit
    flat = R.fit_carreau_yasuda(g, np.full(8, 5.0))
    assert abs(flat["eta0"] - 5.0) < 0.05 and abs(R.carreau_yasuda(0.1, flat["eta0"], flat["eta_inf"], flat["lam"], flat["a"], flat["n"]) - 5.0) < 0.05


def test_shape_constrained_carreau_yasuda_fit_recovers_lambda():
    # with a, n and eta_inf pinned to the generating values, the fit of data
    # drawn from each of the paper's four CY curves (its table, 1 % noise,
    # the rate windows of the 76 x 76 runs) recovers eta0 and the onset time
    # lambda; a curve with lambda twice as large gives a fit twice as large
    from paper_2512_13267_gb300 import rheometry as R
    rng = np.random.default_rng(4)
    table = {4: (13.20, 0.0, 23.50, 0.71, 0.60), 8: (34.29, 3.15, 89.75, 0.95, 0.37),
             16: (173.18, 4.45, 353.48, 0.55, 0.18), 32: (242.83, 4.81, 1307.88, 1.23, 0.29)}
    rates = {4: [0.002, 0.005, 0.01, 0.02, 0.05, 0.1, 0.2],
             8: [0.001, 0.002, 0.005, 0.01, 0.02, 0.05, 0.1],
             16: [0.0005, 0.001, 0.002, 0.005, 0.01, 0.02],
             32: [0.0002, 0.0005, 0.001, 0.002, 0.005, 0.01]}
    for nd, (e0, einf, lam, a, n) in table.items():
        g = np.array(rates[nd])
        for scale in (1.0, 2.0):
            eta = R.carreau_yasuda(g, e0, einf, scale * lam, a, n) * (1 + 0.01 * rng.standard_normal(len(g)))
            fit = R.fit_carreau_yasuda(g, eta, 0.01 * eta, fix_eta_inf=einf, fix_a=a, fix_n=n)
            assert abs(fit["lam"] / (scale * lam) - 1) < 0.15, (nd, scale, fit)
            assert abs(fit["eta0"] / e0 - 1) < 0.1, (nd, scale, fit)
            assert fit["a"] == a and fit["n"] == n and fit["eta_inf"] == einf


def test_relaxation_time_from_decay():
    # a fast (0.3) plus a slow (50) exponential mode with noise: the tail fit
    # past the fast decay finds the slow time constant; a single exponential
    # gives its time constant to both estimators; samples in the noise are
    # left out
    from paper_2512_13267_gb300 import rheometry as R
    rng = np.random.default_rng(3)
    t = np.arange(0.5, 400.0, 1.0)
    se = np.full_like(t, 2e-3)
    g = 0.8 * np.exp(-t / 0.3) + 0.2 * np.exp(-t / 50.0) + rng.normal(scale=2e-3, size=t.size)
    r = R.relaxation_time(t, g, se, t_min=5.0)
    assert abs(r["lam_tail"] - 50.0) < 3 * r["lam_tail_se"] + 1.0, r
    assert r["t_max"] < 260  # stops where g falls into the noise (0.2 e^{-t/50} = 6e-3 near 170)
    one = R.relaxation_time(t, np.exp(-t / 20.0), np.full_like(t, 1e-7))
    assert abs(one["lam_tail"] - 20.0) < 1e-6 and abs(one["lam_moment"] - 20.0) < 0.05
    flat = R.relaxation_time(t, np.full_like(t, 1e-4), np.full_like(t, 1e-3))
    assert np.isnan(flat["lam_tail"])
