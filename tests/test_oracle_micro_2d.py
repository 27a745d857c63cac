"""Pins of the FP64 micro oracle in two dimensions (the paper's melt boxes,
Table 1 parameters): the 2D pair search against brute force, Newton's third
law and zero out-of-plane forces, the fluctuation-dissipation temperature
with two moving axes, the 2D Boltzmann bond distribution of a FENE spring,
the kinetic IK stress per area, and the Lees-Edwards streaming profile."""
import numpy as np
import pytest
from scipy.integrate import quad

import oracle as O
from paper_2512_13267_gb300 import synth as S

ZERO_L = np.zeros(9)
PAPER = dict(a_ij=25.0, gamma=4.5, sigma=3.0, H_fene=50.0, R0=1.5, dt=0.005)


def _params(**kw):
    d = dict(PAPER, dim=2)
    d.update(kw)
    return O.dpd_params(**d)


def _melt(E, nd, seed, L=None, flow="periodic", **kw):
    n = int(round(4 * E * E))
    n -= n % nd
    p, v = S.initial_box_state((E, E, 1.0), n, seed, 0, L=L, flow=flow, dim=2)
    return O.Box((E, E, 1.0), p, v, n_chains=n // nd, chain_len=nd, **kw)


def _block_se(x, nblocks):
    x = np.asarray(x)
    blocks = x[: len(x) // nblocks * nblocks].reshape(nblocks, -1).mean(axis=1)
    return blocks.mean(), blocks.std(ddof=1) / np.sqrt(nblocks)


@pytest.mark.parametrize("flow,L,le", [(O.FLOW_PERIODIC, ZERO_L, 0.0),
                                        (O.FLOW_LEES_EDWARDS, np.array([0, 0.2, 0, 0, 0, 0, 0, 0, 0.0]), 1.7),
                                        (O.FLOW_AFBC, np.array([0.1, 0.4, 0, -0.2, -0.1, 0, 0, 0, 0.0]), 0.0)])
@pytest.mark.parametrize("E", [3.0, 5.5])
def test_2d_cell_list_equals_brute_force(flow, L, le, E):
    par = _params(flow_mode=flow)
    b = _melt(E, 4, 3, step=4, le_offset=le)
    f1, v1, e1 = O.compute_forces(par, b, L, brute=False)
    f2, v2, e2 = O.compute_forces(par, b, L, brute=True)
    assert e1 == 0 and e2 == 0
    assert np.abs(f1 - f2).max() <= 1e-12 * np.abs(f2).max()
    assert np.abs(v1 - v2).max() <= 1e-12 * np.abs(v2).max()
    # in-plane: no z forces, no z virial components
    assert np.all(f1[:, 2] == 0.0) and np.all(v1[[2, 4, 5]] == 0.0)
    # Newton's third law
    assert np.abs(f1.sum(axis=0)).max() <= 1e-11 * np.abs(f1).sum()


def test_2d_pairs_stay_inside_the_plane():
    # one cell layer: a 2D box must not pick up pairs from periodic z images
    par = _params(flow_mode=O.FLOW_PERIODIC, a_ij=25.0, gamma=0.0, sigma=0.0, H_fene=0.0)
    p = np.array([[1.0, 1.0, 0.0], [1.5, 1.0, 0.0]])
    b = O.Box((4.0, 4.0, 1.0), p, np.zeros((2, 3)), n_chains=0, chain_len=2)
    f, _, _ = O.compute_forces(par, b)
    # one pair at r = 0.5: F = a (1 - r) along x, once (a z image would double it)
    assert np.allclose(f[0], [-12.5, 0, 0], atol=1e-12) and np.allclose(f[1], [12.5, 0, 0])


def test_2d_fdt_equilibrium_temperature():
    # sigma^2 = 2 gamma kBT: two moving axes share kBT each (dt = 0.005)
    par = _params(flow_mode=O.FLOW_PERIODIC)
    b = _melt(6.0, 4, 21)
    O.compute_forces(par, b)
    O.advance(par, b, ZERO_L, 400)
    T = []
    for _ in range(60):
        O.advance(par, b, ZERO_L, 25)
        T.append(par.mass * (b.vel[:, :2] ** 2).sum() / (2 * b.n))
    assert np.all(b.vel[:, 2] == 0.0) and np.all(b.pos[:, 2] == 0.0)
    m, se = _block_se(T, 10)
    assert abs(m - 1.0) < max(3 * se, 0.01), (m, se)


def test_2d_fene_bond_length_distribution_ideal_bath():
    # a_ij = 0: a bond vector in the plane is Boltzmann distributed,
    # P(b) ~ b (1 - b^2/R0^2)^(H R0^2 / 2kT) (the 2D measure is b db)
    par = _params(flow_mode=O.FLOW_PERIODIC, a_ij=0.0)
    E, nd = 8.0, 8
    b = _melt(E, nd, 5)
    nch = b.n // nd
    O.compute_forces(par, b)
    O.advance(par, b, ZERO_L, 400)
    b2 = []
    for _ in range(40):
        O.advance(par, b, ZERO_L, 60)
        x = b.pos[: nch * nd, :2].reshape(nch, nd, 2)
        d = np.diff(x, axis=1)
        d -= E * np.rint(d / E)
        b2.append((d ** 2).sum(-1).mean())
    H, R0 = par.H_fene, par.R0
    ex = H * R0 ** 2 / (2 * par.kBT)
    num = quad(lambda x: x ** 3 * (1 - x * x / R0 ** 2) ** ex, 0, R0)[0]
    den = quad(lambda x: x * (1 - x * x / R0 ** 2) ** ex, 0, R0)[0]
    m, se = _block_se(b2, 8)
    assert abs(m - num / den) < 3 * se + 1e-3 * num / den, (m, se, num / den)


def test_2d_kinetic_ik_stress_is_minus_n_kT_per_area():
    # IK kinetic part of an equilibrium ideal gas (a = 0, no bonds):
    # pi_xx = pi_yy = -n kBT / A, pi_xy = 0 (R9 sign, R11 area)
    par = _params(flow_mode=O.FLOW_PERIODIC, a_ij=0.0)
    E = 6.0
    n = int(4 * E * E)
    p, v = S.initial_box_state((E, E, 1.0), n, 9, 0, dim=2)
    b = O.Box((E, E, 1.0), p, v, n_chains=0, chain_len=2)
    O.compute_forces(par, b)
    O.advance(par, b, ZERO_L, 200)
    xs, ys = [], []
    for _ in range(40):
        mean, _, _ = O.advance(par, b, ZERO_L, 25)
        # remove the virial part (dissipative/random pair forces average to 0)
        xs.append(mean[0])
        ys.append(mean[1])
    m, se = _block_se(xs, 8)
    assert abs(m + n / (E * E)) < 3 * se + 0.02 * n / (E * E), (m, se, -n / E ** 2)
    m, se = _block_se(ys, 8)
    assert abs(m + n / (E * E)) < 3 * se + 0.02 * n / (E * E), (m, se, -n / E ** 2)


def test_2d_lees_edwards_linear_streaming_profile():
    gdot = 0.2
    L = np.array([0, gdot, 0, 0, 0, 0, 0, 0, 0.0])
    par = _params(flow_mode=O.FLOW_LEES_EDWARDS)
    E = 8.0
    b = _melt(E, 4, 13, L=L, flow="lees_edwards")
    O.compute_forces(par, b, L)
    O.advance(par, b, L, 400)
    nb = 4
    prof = []
    for _ in range(30):
        O.advance(par, b, L, 40)
        k = np.minimum((b.pos[:, 1] / E * nb).astype(int), nb - 1)
        prof.append([b.vel[k == j, 0].mean() for j in range(nb)])
    prof = np.asarray(prof)
    yc = (np.arange(nb) + 0.5) * E / nb
    m = prof.mean(axis=0)
    se = prof.reshape(6, 5, nb).mean(axis=1).std(axis=0, ddof=1) / np.sqrt(6)
    assert np.all(np.abs(m - gdot * (yc - E / 2)) < 3 * se + 0.02), (m, se)
    mean, _, _ = O.advance(par, b, L, 400)
    assert mean[3] > 0 and mean[2] == 0.0
