"""Sharded micro steps on the GPU: a batch holding boxes lo..hi-1 of a larger
system (one rank's share, lhmm_batch_desc.box_id_offset = lo) draws the
same noise as those boxes do in one batch of the whole system, and the
sharded coupled step (sharding.ShardedCoupled over lhmm.Sph and lhmm.Micro)
reproduces the coupled handle's macro steps.  Several shards run here one
after the other on one GPU; across GPUs the only difference is the stress
all-gather, which tests/test_sharding.py checks on CPU ranks."""
import numpy as np
import pytest

from paper_2512_13267_gb300 import sharding, synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _states(m):
    return [m.get_state(b)[:4] for b in range(m.n_boxes)]


def test_shards_with_box_id_offsets_equal_the_whole_batch():
    from paper_2512_13267_gb300 import lhmm as lh
    n = 7
    batch = S.make_batch(np.full(n, 5.0), S.random_velocity_gradients(n, 9, rate_range=(0.05, 0.5)), 9)
    p = lh.dpd_params(flow="afbc", seed=9)
    whole = lh.Micro.from_batch(p, batch)
    st = torch.zeros((n, 6), dtype=torch.float64, device="cuda")
    whole.advance(torch.from_numpy(batch.L).cuda(), 20, st)
    ref, ref_states = st.cpu().numpy(), _states(whole)
    whole.close()
    for lo, hi in sharding.partition_boxes(batch.n_beads, 3):
        part = batch.boxes(lo, hi)
        m = lh.Micro.from_batch(p, part, box_id_offset=lo)
        s = torch.zeros((hi - lo, 6), dtype=torch.float64, device="cuda")
        m.advance(torch.from_numpy(part.L).cuda(), 20, s)
        assert np.array_equal(s.cpu().numpy(), ref[lo:hi])
        for a, b in zip(_states(m), ref_states[lo:hi]):
            for x, y in zip(a, b):
                assert np.array_equal(np.asarray(x), np.asarray(y))
        m.close()
    # without the offset a shard's boxes draw other noise
    part = batch.boxes(3, n)
    m = lh.Micro.from_batch(p, part)
    s = torch.zeros((n - 3, 6), dtype=torch.float64, device="cuda")
    m.advance(torch.from_numpy(part.L).cuda(), 20, s)
    assert not np.array_equal(s.cpu().numpy(), ref[3:])
    m.close()


class _TwoShards:
    """Two shards of the boxes advanced one after the other on one GPU."""

    def __init__(self, shards, ranges):
        self.shards, self.ranges = shards, ranges

    def advance(self, L):
        return torch.cat([sh.advance(L[lo:hi]) for sh, (lo, hi) in zip(self.shards, self.ranges)])


def test_sharded_coupled_step_equals_coupled_handle():
    from paper_2512_13267_gb300 import lhmm as lh
    cfg, batch = S.coupled_channel(nx=16, ny=8, box_beads=375, U_o=0.25, eta_s=0.1, delta_t=0.1)
    n, M, k = cfg["pos"].shape[0], cfg["substeps"], 10
    sp = lh.sph_params(n, 0, Lx=cfg["Lx"], Ly=cfg["Ly"], h=cfg["h"], mass=cfg["mass"], rho0=1.0,
                       c=cfg["c"], theta_pb=0.1, eta_s=0.1, dt=cfg["dt"],
                       body_force=(cfg["body_force"], 0.0), body_mode=lh.SPH_BODY_REVERSE_POISEUILLE)
    p = lh.dpd_params(flow="afbc", seed=3, alpha=0.05)
    # the coupled handle
    sph = lh.Sph(sp, cfg["pos"], cfg["vel"])
    micro = lh.Micro.from_batch(p, batch)
    cpl = lh.Coupled(sph, micro, M, k)
    cpl.step(3, use_graph=False)
    torch.cuda.synchronize()
    L_ref, st_ref = cpl.exchange()
    ref_pos = sph.get_state()[0]
    cpl.close()
    micro.close()
    sph.close()
    # the sharded driver, two shards of the boxes on this GPU
    sph2 = lh.Sph(sp, cfg["pos"], cfg["vel"])
    ranges = sharding.partition_boxes(batch.n_beads, 2)
    shards = [sharding.GpuMicro(lh.Micro.from_batch(p, batch.boxes(lo, hi), box_id_offset=lo), k)
              for lo, hi in ranges]
    drv = sharding.ShardedCoupled(sharding.GpuSph(sph2, n, M), _TwoShards(shards, ranges),
                                  [(0, n)], torch.zeros((n, 6), dtype=torch.float64, device="cuda"))
    stress = drv.step(3)
    torch.cuda.synchronize()
    assert np.array_equal(sph2.get_state()[0], ref_pos)
    assert np.array_equal(stress.cpu().numpy(), st_ref)
    assert np.array_equal(drv.sph.L.cpu().numpy(), L_ref)
    for sh in shards:
        sh.micro.close()
    sph2.close()
