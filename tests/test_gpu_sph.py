"""GPU parity of the SPH macro step against the FP64 oracle (through the C ABI).

FP32 sums of ~30 neighbour terms: accelerations are compared relative to the
largest pair-term scale of the configuration, velocity gradients relative to
their largest component."""
import numpy as np
import pytest

import oracle as O
from paper_2512_13267_gb300 import synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _lh():
    from paper_2512_13267_gb300 import lhmm
    return lhmm


def _setup(nx=24, ny=16, Lx=1.5, Ly=1.0, jitter=0.15, kernel=0, visc=0, body=(0.05, 0.0),
           body_mode=1, eta=0.1, c=2.0, dt=2e-3, n_wall=0, pos=None, seed=0):
    dh = Ly / ny
    if pos is None:
        pos = S.sph_lattice(nx, ny, Lx, Ly, seed=seed, jitter=jitter)
    n = pos.shape[0]
    rng = np.random.default_rng(seed + 1)
    vel = rng.normal(scale=0.05, size=(n, 2))
    vel[n - n_wall:] = 0.0
    kw = dict(Lx=Lx, Ly=Ly, h=3 * dh, mass=dh * dh, rho0=1.0, c=c, theta_pb=0.1, eta_s=eta,
              zeta_s=0.0, dt=dt, kernel=kernel, visc_coeffs=visc, body_force=body,
              body_mode=body_mode)
    lh = _lh()
    gp = lh.sph_params(n, n_wall, **kw)
    op = O.sph_params(n=n, **kw)
    pos32 = pos.astype(np.float32)
    vel32 = vel.astype(np.float32)
    g = lh.Sph(gp, pos32, vel32)
    is_wall = np.zeros(n, np.int32)
    is_wall[n - n_wall:] = 1
    return g, op, pos32.astype(np.float64), vel32.astype(np.float64), is_wall


def _scale(op, pos, vel):
    # magnitude of the largest single pressure pair term (cancellation scale)
    acc, d = O.sph_accel(op, pos, vel)
    p = np.array([O.sph_pressure(op, op.mass * x) for x in d])
    return np.abs(p / d ** 2).max() * O.sph_F(op.kernel, 0.0, op.h) * op.h / op.mass


@pytest.mark.parametrize("kernel", [0, 1])
def test_initial_accelerations(kernel, parity_report):
    g, op, pos, vel, wall = _setup(kernel=kernel)
    acc_ref, d_ref = O.sph_accel(op, pos, vel, is_wall=wall)
    _, _, acc, d = g.get_state()
    assert np.abs(d - d_ref).max() <= 2e-6 * d_ref.max()
    assert np.abs(acc - acc_ref).max() <= 2e-5 * _scale(op, pos, vel)
    name = "Lucy" if kernel else "Wendland C2"
    parity_report("SPH number density, " + name, np.abs(d - d_ref).max() / d_ref.max(), 2e-6,
                  "max |dd| / max d")
    parity_report("SPH acceleration, " + name,
                  np.abs(acc - acc_ref).max() / _scale(op, pos, vel), 2e-5,
                  "max |da| / largest pressure pair term")
    g.close()


def test_stress_coupling_and_velocity_gradient(parity_report):
    g, op, pos, vel, wall = _setup()
    n = pos.shape[0]
    rng = np.random.default_rng(5)
    st6 = rng.normal(scale=0.3, size=(n, 6))
    st = torch.from_numpy(st6).cuda()
    L = torch.zeros((n, 9), dtype=torch.float32, device="cuda")
    g.recompute_forces(st)
    g.step(0, L_out_dev=L)
    _, _, acc, d = g.get_state()
    stress3 = np.stack([st6[:, 0], st6[:, 3], st6[:, 1]], axis=1)
    acc_ref, d_ref = O.sph_accel(op, pos, vel, is_wall=wall, stress3=stress3)
    assert np.abs(acc - acc_ref).max() <= 2e-5 * _scale(op, pos, vel)
    L_ref = O.sph_velgrad(op, pos, vel, d_ref)
    got = L.cpu().numpy()
    assert np.all(got[:, [2, 5, 6, 7, 8]] == 0)
    got4 = got[:, [0, 1, 3, 4]]
    assert np.abs(got4 - L_ref).max() <= 1e-4 * np.abs(L_ref).max()
    parity_report("SPH acceleration with micro stress", np.abs(acc - acc_ref).max()
                  / _scale(op, pos, vel), 2e-5, "max |da| / largest pressure pair term")
    parity_report("SPH velocity gradient", np.abs(got4 - L_ref).max() / np.abs(L_ref).max(),
                  1e-4, "max |dL| / max |L|")
    g.close()


def test_velocity_verlet_substeps(parity_report):
    g, op, pos, vel, wall = _setup(dt=1e-3)
    acc, _ = O.sph_accel(op, pos, vel, is_wall=wall)
    g.step(40)
    O.sph_steps(op, pos, vel, acc, 40, is_wall=wall)
    p, v, a, d = g.get_state()
    dp = p - pos
    dp -= np.array([op.Lx, op.Ly]) * np.rint(dp / np.array([op.Lx, op.Ly]))
    assert np.abs(dp).max() < 1e-5
    assert np.abs(v - vel).max() < 1e-4 * max(1.0, np.abs(vel).max())
    parity_report("SPH 40 VV substeps, positions", np.abs(dp).max(), 1e-5, "max |dr|")
    parity_report("SPH 40 VV substeps, velocities", np.abs(v - vel).max()
                  / max(1.0, np.abs(vel).max()), 1e-4, "max |dv| / max(1, max |v|)")
    g.close()


def test_walls_stay_fixed_and_push_fluid():
    pos, is_wall, Lbox, dh = S.cylinder_array(n_fluid_target=600, radius_frac=0.25)
    n_wall = int(is_wall.sum())
    g, op, p0, v0, wall = _setup(pos=pos, Lx=Lbox, Ly=Lbox, n_wall=n_wall, body=(0.5, 0.0),
                                 body_mode=0, jitter=0.0, ny=int(round(1 / dh)))
    acc_ref, _ = O.sph_accel(op, p0, v0, is_wall=wall)
    _, _, acc, _ = g.get_state()
    assert np.all(acc[-n_wall:] == 0)
    assert np.abs(acc - acc_ref).max() <= 2e-5 * _scale(op, p0, v0)
    g.step(20)
    p, v, _, _ = g.get_state()
    assert np.array_equal(p[-n_wall:], p0[-n_wall:].astype(np.float32))
    assert np.all(v[-n_wall:] == 0)
    g.close()


def test_reverse_poiseuille_channel_develops_analytic_profile():
    # the channel workload shape (64 x 32 particles) with a Newtonian solvent:
    # steady state within 3 % of the analytic profile away from the kinks
    Ly, ny, nx = 1.0, 32, 64
    dh = Ly / ny
    Lx = nx * dh
    pos = S.sph_lattice(nx, ny, Lx, Ly)
    lh = _lh()
    eta, F = 0.1, 0.16
    p = lh.sph_params(pos.shape[0], 0, Lx=Lx, Ly=Ly, h=3 * dh, mass=dh * dh, rho0=1.0, c=1.0,
                      theta_pb=0.1, eta_s=eta, dt=0.01 * (20 / ny) ** 2, body_force=(F, 0.0),
                      body_mode=lh.SPH_BODY_REVERSE_POISEUILLE)
    g = lh.Sph(p, pos, np.zeros_like(pos))
    g.step(int(round(3.0 / p.dt)))
    q, v, _, _ = g.get_state()
    y = q[:, 1].astype(np.float64)
    k = F / (2 * eta)
    exact = np.where(y < Ly / 2, -k * y * (Ly / 2 - y), k * (y - Ly / 2) * (Ly - y))
    vmax = F * Ly ** 2 / (32 * eta)
    dist = np.minimum.reduce([np.abs(y), np.abs(y - Ly / 2), np.abs(y - Ly)])
    inner = dist > 3 * dh
    assert np.abs(v[inner, 0] - exact[inner]).max() / vmax < 0.03
    g.close()
