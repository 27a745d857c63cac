"""The allocation-free SPH velocity-gradient entry point.

lhmm_sph_velgrad_noalloc serves callers that may not allocate device memory
when they need the gradients; it keeps its scratch in a fixed array inside the
library.  This file runs last (after every other test) so that a failure here
never hides the others.  Two calls in a row, on different particle states,
must each reproduce what the regular entry point (lhmm_sph_step with zero
substeps) returns for the same state."""
import numpy as np
import pytest

from paper_2512_13267_gb300 import synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _state(seed, n_wall=0):
    if n_wall:
        pos, is_wall, Lbox, dh = S.cylinder_array(n_fluid_target=700, radius_frac=0.25)
        Lx = Ly = Lbox
        n_wall = int(is_wall.sum())
    else:
        nx, ny, Lx, Ly = 32, 20, 1.6, 1.0
        dh = Ly / ny
        pos = S.sph_lattice(nx, ny, Lx, Ly, seed=seed, jitter=0.2)
    rng = np.random.default_rng(seed)
    vel = rng.normal(scale=0.1, size=pos.shape)
    if n_wall:
        vel[-n_wall:] = 0.0
    return pos.astype(np.float32), vel.astype(np.float32), Lx, Ly, dh, n_wall


def _params(lh, n, n_wall, Lx, Ly, dh):
    return lh.sph_params(n, n_wall, Lx=Lx, Ly=Ly, h=3 * dh, mass=dh * dh, rho0=1.0, c=2.0,
                         theta_pb=0.1, eta_s=0.1, dt=1e-3)


def test_noalloc_matches_regular_entry_point_on_two_calls():
    from paper_2512_13267_gb300 import lhmm as lh
    for seed, n_wall in ((3, 0), (4, 1)):
        pos, vel, Lx, Ly, dh, nw = _state(seed, n_wall)
        n = pos.shape[0]
        p = _params(lh, n, nw, Lx, Ly, dh)
        ref_h = lh.Sph(p, pos, vel)
        L_ref = torch.zeros((n - nw, 9), dtype=torch.float32, device="cuda")
        ref_h.step(0, L_out_dev=L_ref)
        torch.cuda.synchronize()
        L = torch.full((n - nw, 9), 7.0, dtype=torch.float32, device="cuda")
        lh.sph_velgrad_noalloc(p, torch.from_numpy(pos).cuda(), torch.from_numpy(vel).cuda(), L)
        torch.cuda.synchronize()
        a, b = L.cpu().numpy(), L_ref.cpu().numpy()
        assert np.allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max()), np.abs(a - b).max()
        ref_h.close()


def test_noalloc_bins_positions_outside_the_box_at_their_image():
    # a caller's positions need not lie in [0, L): every particle shifted by
    # whole box lengths (up to three in each direction) must give the in-box
    # result.  Positions on a 2^-16 grid and box lengths 2 and 1 make the
    # shifts, the wrap and the minimum-image distances exact, so the two calls
    # agree bit for bit; both must also match the regular entry point.
    from paper_2512_13267_gb300 import lhmm as lh
    nx, ny, Lx, Ly = 32, 16, 2.0, 1.0
    dh = Ly / ny
    pos = S.sph_lattice(nx, ny, Lx, Ly, seed=5, jitter=0.2)
    pos = np.round(pos * 65536.0) / 65536.0
    pos[:, 0] %= Lx
    pos[:, 1] %= Ly
    rng = np.random.default_rng(5)
    vel = rng.normal(scale=0.1, size=pos.shape)
    k = rng.integers(-3, 4, size=pos.shape)
    shifted = pos + k * np.array([Lx, Ly])
    assert np.abs(k).max() == 3 and (shifted < 0).any() and (shifted[:, 0] >= Lx).any()
    n = pos.shape[0]
    p = _params(lh, n, 0, Lx, Ly, dh)
    vel_d = torch.from_numpy(vel.astype(np.float32)).cuda()
    outs = []
    for x in (pos, shifted):
        L = torch.full((n, 9), 7.0, dtype=torch.float32, device="cuda")
        lh.sph_velgrad_noalloc(p, torch.from_numpy(x.astype(np.float32)).cuda(), vel_d, L)
        torch.cuda.synchronize()
        outs.append(L.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    ref_h = lh.Sph(p, pos.astype(np.float32), vel.astype(np.float32))
    L_ref = torch.zeros((n, 9), dtype=torch.float32, device="cuda")
    ref_h.step(0, L_out_dev=L_ref)
    torch.cuda.synchronize()
    b = L_ref.cpu().numpy()
    ref_h.close()
    assert np.allclose(outs[1], b, rtol=1e-5, atol=1e-6 * np.abs(b).max())


def test_noalloc_rejects_oversize_input():
    from paper_2512_13267_gb300 import lhmm as lh
    n = lh.NOALLOC_MAX_PARTICLES + 1
    p = _params(lh, n, 0, 64.0, 64.0, 0.25)
    x = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    out = torch.zeros((n, 9), dtype=torch.float32, device="cuda")
    with pytest.raises(lh.LhmmError) as ei:
        lh.sph_velgrad_noalloc(p, x, x, out)
    assert ei.value.status == lh.ERR_ARG
