"""Pins of the FP64 micro oracle (DPD + FENE + VV + imposed flow + IK stress).

Each test checks the oracle against something it does not compute itself:
brute-force pair search, Newton's third law, an exact virial identity, the
fluctuation-dissipation temperature, the Boltzmann bond distribution of a
FENE spring, the Lees-Edwards streaming profile, Monte-Carlo bond fractions,
the Table 2 region geometry."""
import numpy as np
import pytest
from scipy.integrate import quad

import oracle as O
from paper_2512_13267_gb300 import synth as S

ZERO_L = np.zeros(9)
SHEAR_L = np.array([0, 0.3, 0, 0, 0, 0, 0, 0, 0.0])
MIXED_L = np.array([0.1, 0.5, 0.0, 0.0, -0.1, 0.2, 0.0, 0.0, 0.0])


def _box(E, seed, n_chains=None, chain_len=10, flow="afbc", L=None, step=0, le=0.0, **kw):
    n = int(round(3 * E ** 3))
    p, v = S.initial_box_state(E, n, seed, 0, L=L, flow=flow)
    nc = n // 20 if n_chains is None else n_chains
    return O.Box(E, p, v, n_chains=nc, chain_len=chain_len, step=step, le_offset=le, **kw)


@pytest.mark.parametrize("flow,L,le", [(O.FLOW_PERIODIC, ZERO_L, 0.0),
                                        (O.FLOW_LEES_EDWARDS, SHEAR_L, 1.234),
                                        (O.FLOW_AFBC, MIXED_L, 0.0)])
@pytest.mark.parametrize("E", [3.0, 4.0, 5.5])
def test_cell_list_equals_brute_force(flow, L, le, E):
    par = O.dpd_params(flow_mode=flow)
    b = _box(E, 7, L=L, le=le, step=5)
    f1, v1, e1 = O.compute_forces(par, b, L, brute=False)
    f2, v2, e2 = O.compute_forces(par, b, L, brute=True)
    assert e1 == 0 and e2 == 0
    scale = np.abs(f2).max()
    assert np.abs(f1 - f2).max() <= 1e-12 * scale
    assert np.abs(v1 - v2).max() <= 1e-12 * np.abs(v2).max()


@pytest.mark.parametrize("flow,L,le", [(O.FLOW_PERIODIC, ZERO_L, 0.0),
                                        (O.FLOW_LEES_EDWARDS, SHEAR_L, 2.5)])
def test_newton_third_law_total_force_zero(flow, L, le):
    par = O.dpd_params(flow_mode=flow)
    b = _box(5.0, 3, L=L, le=le, step=11)
    f, _, _ = O.compute_forces(par, b, L)
    assert np.abs(f.sum(axis=0)).max() <= 1e-12 * np.abs(f).sum()


def test_total_momentum_conserved_periodic():
    par = O.dpd_params(flow_mode=O.FLOW_PERIODIC)
    b = _box(4.0, 9)
    O.compute_forces(par, b)
    p0 = b.vel.sum(axis=0)
    O.advance(par, b, ZERO_L, 300)
    p1 = b.vel.sum(axis=0)
    assert np.abs(p1 - p0).max() < 1e-10


def test_isolated_cluster_virial_identity():
    # For a cluster that touches no periodic image, sum_{i<j} r_ij (x) F_ij
    # equals sum_i r_i (x) F_i exactly (forces are pairwise and central).
    rng = np.random.default_rng(0)
    E, n = 12.0, 300
    p = rng.uniform(4.5, 7.5, size=(n, 3))
    # ten chains of ten beads as random walks with 0.4 steps (bonds < R0)
    steps = rng.normal(size=(10, 9, 3))
    steps *= 0.4 / np.linalg.norm(steps, axis=-1, keepdims=True)
    p[:100] = (rng.uniform(5.5, 6.5, size=(10, 1, 3))
               + np.concatenate([np.zeros((10, 1, 3)), np.cumsum(steps, axis=1)], axis=1)
               ).reshape(100, 3)
    v = rng.normal(size=(n, 3))
    par = O.dpd_params(flow_mode=O.FLOW_PERIODIC)
    b = O.Box(E, p, v, n_chains=10, chain_len=10, step=3)
    f, v6, err = O.compute_forces(par, b)
    assert err == 0
    W = np.einsum("ia,ib->ab", p, f)
    ref = np.array([W[0, 0], W[1, 1], W[2, 2], W[0, 1], W[0, 2], W[1, 2]])
    assert np.allclose(v6, ref, rtol=0, atol=1e-9 * np.abs(W).max())
    assert np.allclose(W, W.T, atol=1e-9 * np.abs(W).max())


def test_ik_stress_of_cluster_has_minus_pressure_sign():
    # pi = -(K + W)/V: a compressed repulsive cluster at rest has W_aa > 0,
    # so the IK normal stresses are negative (a positive pressure)
    rng = np.random.default_rng(1)
    p = rng.uniform(5.0, 7.0, size=(200, 3))
    par = O.dpd_params(flow_mode=O.FLOW_PERIODIC, gamma=0.0, sigma=0.0)
    b = O.Box(12.0, p, np.zeros((200, 3)), n_chains=0, chain_len=10)
    pi6, err = O.ik_sample(par, b)
    f, v6, _ = O.compute_forces(par, b)
    assert err == 0
    assert np.all(pi6[:3] < 0)
    assert np.allclose(pi6, -v6 / 12.0 ** 3)


def test_segment_fraction_matches_monte_carlo():
    rng = np.random.default_rng(4)
    half = np.array([1.0, 0.7, 1.3])
    s = (np.arange(200000) + 0.5) / 200000
    for _ in range(40):
        a = rng.uniform(-2, 2, 3)
        b = a + rng.uniform(-1, 1, 3)
        pts = a[None, :] + s[:, None] * (b - a)[None, :]
        mc = np.mean(np.all(np.abs(pts) < half, axis=1))
        assert abs(O.segment_fraction(a, b, half) - mc) < 2e-5
    # axis-parallel segments and degenerate cases
    assert O.segment_fraction([0, 0, 0], [0.5, 0, 0], half) == 1.0
    assert O.segment_fraction([2, 0, 0], [2, 0.5, 0], half) == 0.0
    assert abs(O.segment_fraction([0.5, 0, 0], [1.5, 0, 0], half) - 0.5) < 1e-15


def test_afbc_regions_follow_table2():
    par = O.dpd_params(flow_mode=O.FLOW_AFBC)
    E = 76.0  # the paper's l_total: core 24, BC 13, buffer 13 (Table 2)
    c = 38.0
    assert O.afbc_region(par, E, [c, c, c]) == 0
    assert O.afbc_region(par, E, [c + 11.9, c, c]) == 0
    assert O.afbc_region(par, E, [c + 12.1, c, c]) == 1
    assert O.afbc_region(par, E, [c, c - 24.9, c + 3]) == 1
    assert O.afbc_region(par, E, [c, c, c + 25.1]) == 2
    assert O.afbc_region(par, E, [0.5, c, c]) == 2


def test_afbc_imposes_linear_velocity_on_bc_shell():
    par = O.dpd_params(flow_mode=O.FLOW_AFBC, lambda_star=2.0)
    E = 8.0
    b = _box(E, 5, L=MIXED_L)
    O.compute_forces(par, b, MIXED_L)
    O.advance(par, b, MIXED_L, 3)
    Lm = 2.0 * MIXED_L.reshape(3, 3)
    reg = np.array([O.afbc_region(par, E, r) for r in b.pos])
    bc = reg == 1
    assert bc.sum() > 100
    target = (b.pos[bc] - 0.5 * E) @ Lm.T
    assert np.allclose(b.vel[bc], target, atol=1e-12)
    # the other regions keep thermal velocities
    assert np.abs(b.vel[reg != 1] - (b.pos[reg != 1] - 0.5 * E) @ Lm.T).std() > 0.5


def test_alpha_lambda_scaling_of_output():
    L = MIXED_L
    outs = []
    for alpha, lam in [(1.0, 1.0), (3.0, 1.0)]:
        par = O.dpd_params(flow_mode=O.FLOW_AFBC, alpha=alpha, lambda_star=lam)
        b = _box(6.0, 2, L=L)
        O.compute_forces(par, b, L)
        m, q, err = O.advance(par, b, L, 5)
        outs.append((m, q))
    assert np.allclose(outs[1][0], 3.0 * outs[0][0], rtol=1e-13, atol=0)
    assert np.allclose(outs[1][1], 9.0 * outs[0][1], rtol=1e-13, atol=0)


@pytest.mark.parametrize("flow", [O.FLOW_AFBC, O.FLOW_LEES_EDWARDS])
def test_lambda_star_scales_input_gradient_and_output_stress(flow):
    # Eq. micro_bc: the box sees lambda* L; Eq. pip: it returns (alpha /
    # lambda*) <pi'>.  A run with (alpha, lambda*) = (3, 2) under L must equal
    # 3/2 x a run with (1, 1) under 2 L: doubling is exact in binary floating
    # point, so both trajectories are the same to the last bit and only the
    # output factor alpha/lambda* = 1.5 remains.  A dropped, inverted or
    # doubled lambda* anywhere fails this.
    L = SHEAR_L if flow == O.FLOW_LEES_EDWARDS else MIXED_L
    fl = "lees_edwards" if flow == O.FLOW_LEES_EDWARDS else "afbc"
    runs = []
    for alpha, lam, Lin in [(3.0, 2.0, L), (1.0, 1.0, 2.0 * L)]:
        par = O.dpd_params(flow_mode=flow, alpha=alpha, lambda_star=lam)
        b = _box(6.0, 2, L=2.0 * L, flow=fl)
        O.compute_forces(par, b, Lin)
        m, q, err = O.advance(par, b, Lin, 8)
        assert err == 0
        runs.append((m, q, b))
    (m1, q1, b1), (m2, q2, b2) = runs
    assert np.array_equal(b1.pos, b2.pos) and np.array_equal(b1.vel, b2.vel)
    assert np.allclose(m1, 1.5 * m2, rtol=1e-15, atol=0)
    assert np.allclose(q1, 2.25 * q2, rtol=1e-15, atol=0)
    # and lambda* = 2 is not lambda* = 1: the dynamics do change
    par = O.dpd_params(flow_mode=flow, alpha=1.0, lambda_star=1.0)
    b = _box(6.0, 2, L=2.0 * L, flow=fl)
    O.compute_forces(par, b, L)
    m3, _, _ = O.advance(par, b, L, 8)
    assert not np.allclose(m3, m2, rtol=1e-6)


def test_3d_kinetic_ik_stress_is_minus_rho_kT():
    # Eq. kinetic_stress in a periodic box at rest: by equipartition the
    # kinetic part sum_i m v_i (x) v_i / V has mean rho kBT on the diagonal and
    # zero off it, for any bead mass (m = 2 here, so a dropped mass factor
    # fails).  The oracle's kinetic part is its IK sample minus its own pair
    # virial, -pi V - W (R9: pi = -(K + W)/V).  dt = 0.01 heats a DPD fluid by
    # about 1 % (reported by the thermostat pin), hence the 1 % floor.
    par = O.dpd_params(flow_mode=O.FLOW_PERIODIC, mass=2.0)
    E = 5.0
    n = int(round(3 * E ** 3))
    p, v = S.initial_box_state(E, n, 17, 0, mass=par.mass)
    b = O.Box(E, p, v, n_chains=n // 20, chain_len=10)
    V = E ** 3
    O.compute_forces(par, b)
    O.advance(par, b, ZERO_L, 800)
    K = []
    for _ in range(160):
        O.advance(par, b, ZERO_L, 20)
        pi6, err = O.ik_sample(par, b)
        _, W, _ = O.compute_forces(par, b)
        assert err == 0
        K.append((-pi6 * V - W) / V)
    K = np.asarray(K)
    rho_kT = b.n * par.kBT / V
    for k in range(6):
        m, se = _block_se(K[:, k], 16)
        target = rho_kT if k < 3 else 0.0
        assert abs(m - target) < max(3 * se, 0.01 * rho_kT), (k, m, se, target)
    # the kinetic part of one sample is the mass-weighted velocity dyadic
    vv = par.mass * np.einsum("ia,ib->ab", b.vel, b.vel) / V
    assert np.allclose(K[-1][[0, 1, 2]], np.diag(vv), rtol=1e-10)


def test_split_advance_is_bitwise_resume():
    par = O.dpd_params(flow_mode=O.FLOW_LEES_EDWARDS)
    b1 = _box(5.0, 8, L=SHEAR_L, flow="lees_edwards")
    b2 = _box(5.0, 8, L=SHEAR_L, flow="lees_edwards")
    for b in (b1, b2):
        O.compute_forces(par, b, SHEAR_L)
    O.advance(par, b1, SHEAR_L, 20)
    O.advance(par, b2, SHEAR_L, 7)
    O.advance(par, b2, SHEAR_L, 13)
    assert np.array_equal(b1.pos, b2.pos) and np.array_equal(b1.vel, b2.vel)
    assert b1.step == b2.step == 20 and b1.le_offset == b2.le_offset


def test_fene_overstretch_is_reported():
    par = O.dpd_params(flow_mode=O.FLOW_PERIODIC)
    p = np.array([[2.0, 2, 2], [3.6, 2, 2], [5, 5, 5], [1, 1, 1]])
    b = O.Box(6.0, p, np.zeros((4, 3)), n_chains=1, chain_len=2)
    _, _, err = O.compute_forces(par, b)
    assert err & O.ERR_BOND_OVERSTRETCH


def _block_se(x, nblocks):
    x = np.asarray(x)
    blocks = x[: len(x) // nblocks * nblocks].reshape(nblocks, -1).mean(axis=1)
    return blocks.mean(), blocks.std(ddof=1) / np.sqrt(nblocks)


def test_fdt_equilibrium_temperature():
    # sigma^2 = 2 gamma kBT fixes the equilibrium temperature (Sec. 2.3)
    par = O.dpd_params(flow_mode=O.FLOW_PERIODIC)
    b = _box(5.0, 21)
    O.compute_forces(par, b)
    O.advance(par, b, ZERO_L, 200)
    T = []
    for _ in range(60):
        O.advance(par, b, ZERO_L, 25)
        T.append(par.mass * (b.vel ** 2).sum() / (3 * b.n))
    m, se = _block_se(T, 10)
    assert abs(m - 1.0) < max(3 * se, 0.01), (m, se)


def test_fene_bond_length_distribution_ideal_bath():
    # a_ij = 0: the bonded pair feels only FENE (+ thermostat), so the bond
    # vector is Boltzmann distributed, P(b) ~ b^2 (1 - b^2/R0^2)^(H R0^2 / 2kT),
    # and bonds are independent: <R_ee^2> = (N_d - 1) <b^2>.
    par = O.dpd_params(flow_mode=O.FLOW_PERIODIC, a_ij=0.0)
    E, nd = 6.0, 10
    n = int(3 * E ** 3)
    nch = n // nd
    p, v = S.initial_box_state(E, n, 5, 0)
    b = O.Box(E, p, v, n_chains=nch, chain_len=nd)
    O.compute_forces(par, b)
    O.advance(par, b, ZERO_L, 300)
    b2, ree = [], []
    for _ in range(40):
        O.advance(par, b, ZERO_L, 60)
        x = b.pos[: nch * nd].reshape(nch, nd, 3)
        d = np.diff(x, axis=1)
        d -= E * np.rint(d / E)
        b2.append((d ** 2).sum(-1).mean())
        ree.append((d.sum(1) ** 2).sum(-1).mean())
    H, R0 = par.H_fene, par.R0
    ex = H * R0 ** 2 / (2 * par.kBT)
    num = quad(lambda x: x ** 4 * (1 - x * x / R0 ** 2) ** ex, 0, R0)[0]
    den = quad(lambda x: x ** 2 * (1 - x * x / R0 ** 2) ** ex, 0, R0)[0]
    b2_th = num / den
    m, se = _block_se(b2, 8)
    assert abs(m - b2_th) < 3 * se + 1e-3 * b2_th, (m, se, b2_th)
    m, se = _block_se(ree, 8)
    assert abs(m - (nd - 1) * b2_th) < 3 * se + 1e-3, (m, se, (nd - 1) * b2_th)


def test_lees_edwards_linear_streaming_profile():
    gdot = 0.5
    L = np.array([0, gdot, 0, 0, 0, 0, 0, 0, 0.0])
    par = O.dpd_params(flow_mode=O.FLOW_LEES_EDWARDS)
    E = 6.0
    b = _box(E, 13, L=L, flow="lees_edwards")
    O.compute_forces(par, b, L)
    O.advance(par, b, L, 200)
    nb = 6
    prof = []
    for _ in range(30):
        O.advance(par, b, L, 40)
        k = np.minimum((b.pos[:, 1] / E * nb).astype(int), nb - 1)
        prof.append([b.vel[k == j, 0].mean() for j in range(nb)])
    prof = np.asarray(prof)
    yc = (np.arange(nb) + 0.5) * E / nb
    target = gdot * (yc - E / 2)
    m = prof.mean(axis=0)
    se = prof.reshape(6, 5, nb).mean(axis=1).std(axis=0, ddof=1) / np.sqrt(6)
    assert np.all(np.abs(m - target) < 3 * se + 0.02), (m, target, se)
    # and the shear stress the IK formula returns is positive (eta_p > 0)
    mean, _, _ = O.advance(par, b, L, 400)
    assert mean[3] > 0


@pytest.mark.parametrize("K,expected", [(0, 30.0), (1, 12.5), (2, 2.5), (3, 0.0)])
def test_bond_exclusion_depth(K, expected):
    # beads 0..3 form one chain on a line at spacing 0.3 (all within rc):
    # the conservative force on bead 0 sums a (1 - r) over the pairs that the
    # exclusion depth K keeps (r = 0.3, 0.6, 0.9 for 1, 2, 3 bonds apart)
    par = O.dpd_params(flow_mode=O.FLOW_PERIODIC, gamma=0.0, sigma=0.0, H_fene=0.0,
                       exclude_bonds=K)
    x = np.array([[1.0 + 0.3 * k, 2.0, 2.0] for k in range(4)])
    b = O.Box(5.0, x, np.zeros((4, 3)), n_chains=1, chain_len=4)
    f, _, err = O.compute_forces(par, b)
    assert err == 0
    assert abs(f[0, 0] + expected) < 1e-12 and abs(f[0, 1]) < 1e-12
    assert np.abs(f.sum(axis=0)).max() < 1e-12


def test_bond_exclusion_stops_at_chain_ends():
    # two 2-bead chains: ids 1 and 2 are consecutive but in different chains,
    # so even K = 3 keeps their pair force; dpd_on_bonded = 0 means K >= 1
    par = O.dpd_params(flow_mode=O.FLOW_PERIODIC, gamma=0.0, sigma=0.0, H_fene=0.0,
                       dpd_on_bonded=0)
    x = np.array([[1.0, 2.0, 2.0], [1.3, 2.0, 2.0], [1.6, 2.0, 2.0], [1.9, 2.0, 2.0]])
    b = O.Box(5.0, x, np.zeros((4, 3)), n_chains=2, chain_len=2)
    f, _, _ = O.compute_forces(par, b)
    # bead 1: pairs (1,0) excluded, (1,2) r = 0.3 kept, (1,3) r = 0.6 kept
    assert abs(f[1, 0] - (-25.0 * 0.7 - 25.0 * 0.4)) < 1e-12
    par3 = O.dpd_params(flow_mode=O.FLOW_PERIODIC, gamma=0.0, sigma=0.0, H_fene=0.0,
                        exclude_bonds=3)
    f3, _, _ = O.compute_forces(par3, b)
    assert np.array_equal(f3, f)


@pytest.mark.parametrize("dim", [3, 2])
def test_afbc_peculiar_mode_keeps_shell_thermal_and_imposes_cell_means(dim):
    # afbc_mode = 1 (R8's alternative): every BC bead gets v = L r' + (v -
    # mean of the BC beads of its cell): per cell the BC beads' mean velocity
    # relative to the imposed field is zero, their spread about it is thermal;
    # positions and the other beads' velocities match afbc_mode = 0
    L = np.array([0.2, 0.5, 0.0, 0.0, -0.2, 0.0, 0.0, 0.0, 0.0])
    E = 9.0
    if dim == 3:
        edge, n = (E, E, E), int(round(3 * E ** 3))
    else:
        edge, n = (E, E, 1.0), int(round(4 * E * E))
    p0, v0 = S.initial_box_state(edge, n, 3, 0, L=L, dim=dim)
    boxes = {}
    for mode in (0, 1):
        par = O.dpd_params(flow_mode=O.FLOW_AFBC, afbc_mode=mode, dim=dim)
        b = O.Box(edge, p0, v0, n_chains=n // 20, chain_len=10)
        O.compute_forces(par, b, L)
        O.advance(par, b, L, 1)
        boxes[mode] = (b, par)
    b0, par0 = boxes[0]
    b1, _ = boxes[1]
    assert np.array_equal(b0.pos, b1.pos)
    reg = np.array([O.afbc_region(par0, edge, b1.pos[i]) for i in range(n)])
    assert np.array_equal(b0.vel[reg != 1], b1.vel[reg != 1])
    u = (b1.pos - 0.5 * np.array(edge)) @ L.reshape(3, 3).T
    nc = [int(np.floor(e)) for e in edge]
    if dim == 2:
        nc[2] = 1
    wf = np.array([e / k for e, k in zip(edge, nc)], np.float64)
    ci = np.minimum(np.floor(b1.pos / wf).astype(int), np.array(nc) - 1)
    cell = ci[:, 0] + nc[0] * (ci[:, 1] + nc[1] * ci[:, 2])
    d = (b1.vel - u)[reg == 1]
    cb = cell[reg == 1]
    for c in np.unique(cb):
        assert np.abs(d[cb == c].mean(axis=0)).max() < 1e-12
    moving = 3 if dim == 3 else 2
    assert d[:, :moving].var() > 0.3  # thermal, not frozen
    assert np.abs((b0.vel - u)[reg == 1]).max() < 1e-12  # mode 0: exact overwrite


def test_diagnostic_potentials_closed_forms():
    # two solvent beads at r = 0.4: U = a rc/2 (1 - r/rc)^2 = 12.5 * 0.36;
    # a 2-bead chain at r = 0.9 adds the FENE energy -H R0^2/2 ln(1 - r^2/R0^2)
    par = O.dpd_params(flow_mode=O.FLOW_PERIODIC)
    x = np.array([[1.0, 2.0, 2.0], [1.4, 2.0, 2.0]])
    v = np.array([[0.5, -1.0, 0.0], [0.1, 0.2, 0.3]])
    out, err = O.diagnostics(par, O.Box(5.0, x, v, n_chains=0, chain_len=2))
    assert err == 0
    assert np.allclose(out[:3], [0.6, -0.8, 0.3], rtol=0, atol=1e-15)
    assert abs(out[3] - 0.5 * (1.25 + 0.14)) < 1e-15
    assert abs(out[4] - 4.5) < 1e-13 and out[5] == 0.0
    x = np.array([[4.6, 2.0, 2.0], [0.5, 2.0, 2.0]])  # 0.9 apart through the x boundary
    out, err = O.diagnostics(par, O.Box(5.0, x, np.zeros((2, 3)), n_chains=1, chain_len=2))
    assert abs(out[4] - 12.5 * 0.01) < 1e-12
    assert abs(out[5] + 0.5 * 30.0 * 2.25 * np.log(1 - 0.81 / 2.25)) < 1e-12
    assert abs(out[6] - out[3] - out[4] - out[5]) < 1e-12


def test_energy_conserved_without_thermostat_to_second_order_in_dt():
    # gamma = sigma = 0: Eq. motion is Hamiltonian with the potentials of the
    # diagnostic, so velocity-Verlet keeps the total energy up to an O(dt^2)
    # error that does not drift.  The forces and the potentials are written
    # separately; a sign or factor mistake in either breaks this.
    errs = []
    for dt in (0.004, 0.002):
        par = O.dpd_params(flow_mode=O.FLOW_PERIODIC, gamma=0.0, sigma=0.0, dt=dt)
        b = _box(4.0, 23)
        O.compute_forces(par, b)
        d0 = O.diagnostics(par, b)[0]
        e0 = d0[6]
        dev = []
        for _ in range(20):
            O.advance(par, b, ZERO_L, int(round(0.02 / dt)))
            d, err = O.diagnostics(par, b)
            assert err == 0
            dev.append(d[6] - e0)
        errs.append(np.abs(dev).max())
        assert np.abs(O.diagnostics(par, b)[0][:3] - d0[:3]).max() < 1e-10  # momentum kept
    # halving dt quarters the energy error (2nd order), within 30 %
    assert 2.8 < errs[0] / errs[1] < 5.2, errs
    assert errs[0] < 2e-3 * b.n
