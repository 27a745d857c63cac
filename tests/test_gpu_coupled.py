"""GPU parity of the coupled macro step (SPH -> grad v -> DPD boxes -> IK stress
-> SPH) against the FP64 oracles, and CUDA-graph replay against eager launch."""
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


def _small_coupled(seed=7, nx=8, ny=8, Ly=1.0, box_edge=4.0, F=0.3, eta=0.2, c=2.0, dt=0.01):
    dh = Ly / ny
    Lx = nx * dh
    pos = S.sph_lattice(nx, ny, Lx, Ly, seed=seed, jitter=0.1).astype(np.float32)
    vel = (np.random.default_rng(seed).normal(scale=0.05, size=pos.shape)).astype(np.float32)
    n = pos.shape[0]
    batch = S.make_batch(np.full(n, box_edge), np.zeros((n, 9), np.float32), seed, flow="afbc")
    sph_kw = dict(Lx=Lx, Ly=Ly, h=3 * dh, mass=dh * dh, rho0=1.0, c=c, theta_pb=0.1, eta_s=eta,
                  zeta_s=0.0, dt=dt, kernel=0, visc_coeffs=0, body_force=(F, 0.0), body_mode=1)
    return pos, vel, batch, sph_kw


def _gpu(pos, vel, batch, sph_kw, alpha, M, k):
    from paper_2512_13267_gb300 import lhmm as lh
    sph = lh.Sph(lh.sph_params(pos.shape[0], 0, **sph_kw), pos, vel)
    micro = lh.Micro.from_batch(lh.dpd_params(flow="afbc", seed=5, alpha=alpha), batch)
    return lh.Coupled(sph, micro, M, k)


def test_two_macro_steps_match_oracle():
    M, k, alpha = 5, 10, 0.05
    pos, vel, batch, sph_kw = _small_coupled()
    cpl = _gpu(pos, vel, batch, sph_kw, alpha, M, k)
    # oracle side
    op = O.sph_params(n=pos.shape[0], **sph_kw)
    mp = O.dpd_params(flow_mode=O.FLOW_AFBC, seed=5, alpha=alpha)
    p = pos.astype(np.float64)
    v = vel.astype(np.float64)
    acc, _ = O.sph_accel(op, p, v)
    boxes = []
    for b in range(batch.n_boxes):
        sl = batch.box_slice(b)
        ob = O.Box(batch.edges[b], batch.pos[sl], batch.vel[sl], int(batch.n_chains[b]),
                   batch.chain_len, box_id=b)
        O.compute_forces(mp, ob, np.zeros(9))
        boxes.append(ob)
    stress6 = np.zeros((batch.n_boxes, 6))
    for step in range(2):
        stress3 = np.stack([stress6[:, 0], stress6[:, 3], stress6[:, 1]], axis=1)
        O.sph_steps(op, p, v, acc, M, stress3=stress3)
        d = O.sph_density(op, p)
        L4 = O.sph_velgrad(op, p, v, d)
        L9 = np.zeros((batch.n_boxes, 9))
        L9[:, [0, 1, 3, 4]] = L4
        stress6, _, st, _ = O.advance_batch(mp, boxes, L9, k)
        assert np.all(st == 0)
        cpl.step(1, use_graph=False)
        Lg, sg = cpl.exchange()
        tolL = (1e-4 if step == 0 else 2e-3) * np.abs(L9).max()
        assert np.abs(Lg - L9).max() <= tolL, (step, np.abs(Lg - L9).max(), tolL)
        scale = 1.0 + np.abs(stress6).max()
        assert np.abs(sg - stress6).max() <= 2e-2 * scale, (step, np.abs(sg - stress6).max())
    cpl.close()


def test_graph_replay_equals_eager():
    M, k, alpha = 4, 6, 0.05
    pos, vel, batch, sph_kw = _small_coupled(seed=9)
    a = _gpu(pos, vel, batch, sph_kw, alpha, M, k)
    b = _gpu(pos, vel, batch, sph_kw, alpha, M, k)
    a.step(4, use_graph=False)
    b.step(4, use_graph=True)  # eager, capture, replay, replay
    La, sa = a.exchange()
    Lb, sb = b.exchange()
    assert np.array_equal(La, Lb) and np.array_equal(sa, sb)
    pa = a.sph.get_state()[0]
    pb = b.sph.get_state()[0]
    assert np.array_equal(pa, pb)
    assert np.array_equal(a.micro.get_state(3)[0], b.micro.get_state(3)[0])
    a.close()
    b.close()


def test_coupled_rejects_mismatched_handles():
    from paper_2512_13267_gb300 import lhmm as lh
    pos, vel, batch, sph_kw = _small_coupled()
    sph = lh.Sph(lh.sph_params(pos.shape[0], 0, **sph_kw), pos, vel)
    small = S.make_batch(np.full(3, 4.0), np.zeros((3, 9), np.float32), 1)
    micro = lh.Micro.from_batch(lh.dpd_params(flow="afbc"), small)
    with pytest.raises(lh.LhmmError):
        lh.Coupled(sph, micro, 2, 2)
