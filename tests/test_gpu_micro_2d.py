"""GPU parity of the planar (dim = 2) micro engine against the FP64 oracle:
the paper's melt boxes (Table 1 parameters, number density 4 per area, all
beads in chains).  Same tolerances as the 3D tests: single-step forces
max |dF| <= 1e-4, 50-step positions <= 1e-3, time-averaged stresses within
3 combined block standard errors."""
import numpy as np
import pytest

import oracle as O
from paper_2512_13267_gb300 import synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PAPER = dict(a_ij=25.0, gamma=4.5, sigma=3.0, H_fene=50.0, R0=1.5, dt=0.005)
FLOW_O = {"periodic": O.FLOW_PERIODIC, "lees_edwards": O.FLOW_LEES_EDWARDS, "afbc": O.FLOW_AFBC}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _batch(flow, seed, nd=8):
    edges = np.array([3.0, 5.0, 8.0, 12.0, 20.0])
    B = len(edges)
    if flow == "lees_edwards":
        L = np.zeros((B, 9), np.float32)
        L[:, 1] = np.array([0.05, 0.1, 0.2, 0.3, 0.5])
    elif flow == "afbc":
        L = S.random_velocity_gradients(B, seed, rate_range=(0.05, 0.5))
        L = L.reshape(B, 3, 3)
        L[:, 2, :] = 0.0
        L[:, :, 2] = 0.0  # the planar flow of an SPH particle
        L = L.reshape(B, 9)
    else:
        L = np.zeros((B, 9), np.float32)
    n = np.rint(4 * edges * edges).astype(int)
    n -= n % nd
    return S.make_batch(edges, L, seed, flow=flow, chain_len=nd, fraction=1.0, n_beads=n, dim=2)


def _pair(batch, flow, seed):
    from paper_2512_13267_gb300 import lhmm as lh
    gp = lh.dpd_params(flow=flow, seed=seed, dim=2, **PAPER)
    op = O.dpd_params(flow_mode=FLOW_O[flow], seed=seed, dim=2, **PAPER)
    m = lh.Micro.from_batch(gp, batch)
    boxes = []
    for b in range(batch.n_boxes):
        sl = batch.box_slice(b)
        ob = O.Box(batch.edges[b], batch.pos[sl], batch.vel[sl], int(batch.n_chains[b]),
                   batch.chain_len, box_id=b)
        O.compute_forces(op, ob, batch.L[b])
        boxes.append(ob)
    return m, op, boxes


def _minimage(d, E):
    return d - E * np.rint(d / E)


@pytest.mark.parametrize("flow", ["periodic", "lees_edwards", "afbc"])
def test_2d_initial_forces_match_oracle(flow, parity_report):
    batch = _batch(flow, 3)
    m, op, boxes = _pair(batch, flow, 3)
    worst = 0.0
    for b, ob in enumerate(boxes):
        pos, vel, f, step, _ = m.get_state(b)
        assert np.all(f[:, 2] == 0.0) and np.all(pos[:, 2] == 0.0)
        assert np.abs(f - ob.force).max() <= 1e-4, (b, np.abs(f - ob.force).max())
        worst = max(worst, np.abs(f - ob.force).max())
    parity_report("2D initial forces, " + flow, worst, 1e-4, "max |dF|")
    m.close()


@pytest.mark.parametrize("flow", ["periodic", "lees_edwards", "afbc"])
def test_2d_fifty_step_trajectory(flow, parity_report):
    # positions within 1e-3; 50-step stress averages within 3 SEs of the
    # oracle's (SE from its per-step samples), second moments within 2 %
    batch = _batch(flow, 8)
    m, op, boxes = _pair(batch, flow, 9)
    L = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    sq = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    m.advance(L, 50, st, stress_sq_dev=sq)
    m.sync()
    got, got_sq = st.cpu().numpy(), sq.cpu().numpy()
    w_pos, w_se = 0.0, 0.0
    for b, ob in enumerate(boxes):
        ref, ref_sq, err = O.advance(op, ob, batch.L[b], 50)
        assert err == 0
        pos, vel, f, step, _ = m.get_state(b)
        assert step == 50 and np.all(pos[:, 2] == 0.0) and np.all(vel[:, 2] == 0.0)
        dpos = np.abs(_minimage(pos - ob.pos, batch.edges[b][0])).max()
        assert dpos <= 1e-3, (b, dpos)
        se = np.sqrt(np.maximum(ref_sq - ref * ref, 0.0) / 50)
        d = np.abs(got[b] - ref)
        assert np.all(d <= 3 * se + 1e-12 * (1 + np.abs(ref))), (b, got[b], ref, se)
        assert np.abs(got_sq[b] - ref_sq).max() <= 2e-2 * (1.0 + np.abs(ref_sq).max())
        assert got[b][2] == 0.0 and got[b][4] == 0.0 and got[b][5] == 0.0
        w_pos = max(w_pos, dpos)
        w_se = max(w_se, float(np.max(np.where(se > 0, d / np.where(se > 0, se, 1), 0))))
    parity_report("2D 50-step positions, " + flow, w_pos, 1e-3, "max |dr|")
    parity_report("2D 50-step stress average, " + flow, w_se, 3.0, "max |dpi| / SE")
    m.close()


def test_2d_block_averaged_shear_stress_of_a_melt():
    # a 12 x 12 melt of N_d = 4 chains under shear 0.05, 30 calls of 200
    # steps: GPU and oracle block means within 3 combined SEs
    batch = S.melt_rheometer_batch(4, [0.05], 1, edge=12.0, seed=4)
    m, op, boxes = _pair(batch, "lees_edwards", 4)
    L = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((1, 6), dtype=torch.float64, device="cuda")
    g_blocks, o_blocks = [], []
    for _ in range(30):
        m.advance(L, 200, st)
        g_blocks.append(st.cpu().numpy()[0].copy())
        ref, _, _ = O.advance(op, boxes[0], batch.L[0], 200)
        o_blocks.append(ref)
    m.sync()
    g = np.asarray(g_blocks)[5:]
    o = np.asarray(o_blocks)[5:]
    se = np.sqrt(g.var(axis=0, ddof=1) / len(g) + o.var(axis=0, ddof=1) / len(o))
    diff = np.abs(g.mean(axis=0) - o.mean(axis=0))
    assert np.all(diff <= 3 * se + 1e-6), (g.mean(0), o.mean(0), se)
    assert g.mean(axis=0)[3] > 0
    m.close()


def test_2d_rejects_bad_dim():
    from paper_2512_13267_gb300 import lhmm as lh
    batch = _batch("periodic", 1)
    with pytest.raises(lh.LhmmError):
        lh.Micro.from_batch(lh.dpd_params(flow="periodic", dim=4, **PAPER), batch)


@pytest.mark.parametrize("K", [1, 3])
def test_2d_bond_exclusion_matches_oracle(K):
    # DPD pairs of one chain up to K bonds apart skipped on both sides
    from paper_2512_13267_gb300 import lhmm as lh
    batch = _batch("lees_edwards", 12, nd=4)
    gp = lh.dpd_params(flow="lees_edwards", seed=5, dim=2, exclude_bonds=K, **PAPER)
    op = O.dpd_params(flow_mode=O.FLOW_LEES_EDWARDS, seed=5, dim=2, exclude_bonds=K, **PAPER)
    m = lh.Micro.from_batch(gp, batch)
    L = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    boxes = []
    for b in range(batch.n_boxes):
        sl = batch.box_slice(b)
        ob = O.Box(batch.edges[b], batch.pos[sl], batch.vel[sl], int(batch.n_chains[b]),
                   batch.chain_len, box_id=b)
        O.compute_forces(op, ob, batch.L[b])
        _, _, f, _, _ = m.get_state(b)
        assert np.abs(f - ob.force).max() <= 1e-4, (b, np.abs(f - ob.force).max())
        boxes.append(ob)
    m.advance(L, 50, st)
    m.sync()
    for b, ob in enumerate(boxes):
        O.advance(op, ob, batch.L[b], 50)
        pos, _, _, _, _ = m.get_state(b)
        assert np.abs(_minimage(pos - ob.pos, batch.edges[b][0])).max() <= 1e-3
    m.close()


def test_2d_afbc_peculiar_mode_matches_oracle(parity_report):
    # R8's alternative on the GPU: each step's AFBC update (BC beads keep
    # their velocity about their cell's BC mean) against the oracle, restarted
    # from the GPU state before every step
    from afbc_steps import stepwise_afbc_parity
    from paper_2512_13267_gb300 import lhmm as lh
    batch = _batch("afbc", 23)
    gp = lh.dpd_params(flow="afbc", seed=23, dim=2, afbc_mode=1, **PAPER)
    op = O.dpd_params(flow_mode=O.FLOW_AFBC, seed=23, dim=2, afbc_mode=1, **PAPER)
    m = lh.Micro.from_batch(gp, batch)
    skipped = stepwise_afbc_parity(m, op, batch, 50, dim=2)
    assert skipped <= 10
    parity_report("thermal-shell AFBC one-step map, 50 steps, 2D", skipped, 10,
                  "bead velocities left out as ambiguous")
    for b in range(batch.n_boxes):
        _, vel, _, _, _ = m.get_state(b)
        assert np.all(vel[:, 2] == 0.0)
    m.close()


def _run_schedule(m, op, boxes, batch, schedule, parity_report, name):
    # each (L, steps) of the schedule advances both sides; positions after
    # every segment within 1e-3, the segment's stress average within 3 SEs
    # of the oracle's per-step samples
    w_pos, w_se = 0.0, 0.0
    for Lseg, steps in schedule:
        Ld = torch.from_numpy(np.ascontiguousarray(Lseg, np.float32)).cuda()
        st = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
        m.advance(Ld, steps, st)
        m.sync()
        got = st.cpu().numpy()
        for b, ob in enumerate(boxes):
            ref, ref_sq, err = O.advance(op, ob, Lseg[b], steps)
            assert err == 0
            pos = m.get_state(b)[0]
            dpos = np.abs(_minimage(pos - ob.pos, batch.edges[b][0])).max()
            assert dpos <= 1e-3, (name, b, dpos)
            se = np.sqrt(np.maximum(ref_sq - ref * ref, 0.0) / steps)
            d = np.abs(got[b] - ref)
            assert np.all(d <= 3 * se + 1e-12 * (1 + np.abs(ref))), (name, b, got[b], ref, se)
            w_pos = max(w_pos, dpos)
            w_se = max(w_se, float(np.max(np.where(se > 0, d / np.where(se > 0, se, 1), 0))))
    parity_report(name + ", positions", w_pos, 1e-3, "max |dr|")
    parity_report(name + ", stress average", w_se, 3.0, "max |dpi| / SE")


def test_2d_stress_relaxation_step_change_matches_oracle(parity_report):
    # the recovery test's schedule (Sec. 5.2): Lees-Edwards shear, then the
    # shear removed (L = 0) while the stress relaxes, then sheared again at
    # another rate; every change of L lands between calls as in the rheometer
    batch = _batch("lees_edwards", 31)
    m, op, boxes = _pair(batch, "lees_edwards", 31)
    L1 = batch.L.copy()
    L0 = np.zeros_like(L1)
    L2 = L1.copy()
    L2[:, 1] *= -0.5
    _run_schedule(m, op, boxes, batch, [(L1, 20), (L0, 15), (L2, 15)], parity_report,
                  "2D shear - rest - reversed shear (Lees-Edwards)")
    m.close()


def test_2d_planar_extension_matches_oracle(parity_report):
    # steady planar extension L = diag(e, -e) through the AFBC shell (the
    # rheometer of rheometry.planar_extension), then the flow stopped
    batch = _batch("afbc", 37)
    e = np.array([0.05, 0.1, 0.2, 0.3, 0.5], np.float32)
    L = np.zeros((batch.n_boxes, 9), np.float32)
    L[:, 0], L[:, 4] = e, -e
    batch.L[:] = L
    m, op, boxes = _pair(batch, "afbc", 37)
    _run_schedule(m, op, boxes, batch, [(L, 25), (np.zeros_like(L), 15)], parity_report,
                  "2D planar extension - rest (AFBC)")
    m.close()


def test_2d_afbc_recovery_schedule_matches_oracle(parity_report):
    # the recovery test in the paper's rheometer (rheometry.stress_relaxation
    # with rheometer="afbc"): simple shear through the AFBC shell, then
    # L = 0, which holds the shell at rest while the core relaxes
    batch = _batch("afbc", 41)
    L = np.zeros((batch.n_boxes, 9), np.float32)
    L[:, 1] = np.array([0.05, 0.1, 0.2, 0.3, 0.5], np.float32)[:batch.n_boxes]
    batch.L[:] = L
    m, op, boxes = _pair(batch, "afbc", 41)
    _run_schedule(m, op, boxes, batch, [(L, 25), (np.zeros_like(L), 20)], parity_report,
                  "2D shear - rest (AFBC recovery)")
    m.close()
