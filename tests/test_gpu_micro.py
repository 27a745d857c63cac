"""GPU parity of the batched micro engine against the FP64 oracle.

All calls go through the C ABI (ctypes binding).  Tolerances: single-step
forces max |dF| <= 1e-4, 50-step positions <= 1e-3, time-averaged stresses
within 3 combined block standard errors."""
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


FLOW_O = {"periodic": O.FLOW_PERIODIC, "lees_edwards": O.FLOW_LEES_EDWARDS, "afbc": O.FLOW_AFBC}


def _pair(batch, flow, seed, **kw):
    lh = _lh()
    gp = lh.dpd_params(flow=flow, seed=seed, **kw)
    op = O.dpd_params(flow_mode=FLOW_O[flow], seed=seed, **kw)
    m = lh.Micro.from_batch(gp, batch)
    boxes = []
    for b in range(batch.n_boxes):
        sl = batch.box_slice(b)
        ob = O.Box(batch.edges[b], batch.pos[sl], batch.vel[sl], int(batch.n_chains[b]),
                   batch.chain_len, box_id=b)
        O.compute_forces(op, ob, batch.L[b])
        boxes.append(ob)
    return m, op, boxes


def _ragged_afbc_batch(seed=5):
    edges = np.array([3.0, 4.0, 5.0, 6.0, 7.5, 9.0, 12.0])
    L = S.random_velocity_gradients(len(edges), seed, rate_range=(0.05, 1.0))
    return S.make_batch(edges, L, seed, flow="afbc")


def _minimage(d, E):
    return d - E * np.rint(d / E)


@pytest.mark.parametrize("flow,lam", [("afbc", 1.0), ("periodic", 1.0), ("lees_edwards", 1.0),
                                      ("afbc", 2.0), ("lees_edwards", 2.0)])
def test_initial_forces_match_oracle(flow, lam, parity_report):
    # lam = lambda*: the boxes see lambda* L (Eq. micro_bc); under Lees-Edwards
    # the sliding images' velocity jump, under AFBC the streaming velocity of
    # the dissipative force's reference, both scale with it
    batch = _ragged_afbc_batch()
    if flow == "lees_edwards":
        batch.L[:] = 0.0
        batch.L[:, 1] = 0.4
    m, op, boxes = _pair(batch, flow, seed=3, lambda_star=lam)
    worst = 0.0
    for b, ob in enumerate(boxes):
        pos, vel, f, step, _ = m.get_state(b)
        assert step == 0
        assert np.abs(f - ob.force).max() <= 1e-4, (b, np.abs(f - ob.force).max())
        assert np.abs(_minimage(pos - ob.pos, batch.edges[b][0])).max() < 1e-5
        worst = max(worst, np.abs(f - ob.force).max())
    parity_report("initial forces, %s, lambda*=%g" % (flow, lam), worst, 1e-4, "max |dF|")
    m.close()


def test_config0_single_box_forces_and_one_step_stress():
    batch = S.single_shear_box(seed=1)
    m, op, boxes = _pair(batch, "lees_edwards", seed=1)
    _, _, f, _, _ = m.get_state(0)
    assert np.abs(f - boxes[0].force).max() <= 1e-4
    L = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((1, 6), dtype=torch.float64, device="cuda")
    m.advance(L, 1, st)
    m.sync()
    ref, _, _ = O.advance(op, boxes[0], batch.L[0], 1)
    got = st.cpu().numpy()[0]
    # one IK sample: sum of ~10^4 FP32 pair terms of size <= ~100 over V = 1000
    assert np.abs(got - ref).max() <= 2e-4, (got, ref)
    _, _, f1, step, le = m.get_state(0)
    assert step == 1 and abs(le - boxes[0].le_offset) < 1e-6
    assert np.abs(f1 - boxes[0].force).max() <= 1e-4
    m.close()


@pytest.mark.parametrize("flow,lam,alpha", [("afbc", 1.0, 1.0), ("lees_edwards", 1.0, 1.0),
                                            ("periodic", 1.0, 1.0), ("afbc", 2.0, 3.0),
                                            ("lees_edwards", 2.0, 3.0)])
def test_fifty_step_trajectory(flow, lam, alpha, parity_report):
    # positions after 50 steps within 1e-3; the 50-step averages of the IK
    # stress (Eq. pip: scaled by alpha/lambda*) within 3 standard errors of
    # the oracle's, the SE taken from the oracle's own per-step samples
    # (stress_sq - stress^2 over 50 samples; consecutive samples are
    # correlated, so this SE is small and the bound strict); the second
    # moments stress_sq within 2 % of their scale
    batch = _ragged_afbc_batch(seed=8)
    if flow == "lees_edwards":
        batch.L[:] = 0.0
        batch.L[:, 1] = 0.5
    m, op, boxes = _pair(batch, flow, seed=9, lambda_star=lam, alpha=alpha)
    L = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    sq = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    m.advance(L, 50, st, stress_sq_dev=sq)
    m.sync()
    got, got_sq = st.cpu().numpy(), sq.cpu().numpy()
    w_pos, w_se, w_sq = 0.0, 0.0, 0.0
    for b, ob in enumerate(boxes):
        ref, ref_sq, err = O.advance(op, ob, batch.L[b], 50)
        assert err == 0
        pos, vel, f, step, _ = m.get_state(b)
        assert step == 50
        dpos = np.abs(_minimage(pos - ob.pos, batch.edges[b][0])).max()
        assert dpos <= 1e-3, (b, dpos)
        se = np.sqrt(np.maximum(ref_sq - ref * ref, 0.0) / 50)
        d = np.abs(got[b] - ref)
        # boxes of edge 3 have an empty AFBC core (zero stress, zero SE)
        assert np.all(d <= 3 * se + 1e-12 * (1 + np.abs(ref))), (b, got[b], ref, se)
        dq = np.abs(got_sq[b] - ref_sq).max()
        assert dq <= 2e-2 * (1.0 + np.abs(ref_sq).max()), (b, got_sq[b], ref_sq)
        w_pos = max(w_pos, dpos)
        w_se = max(w_se, float(np.max(np.where(se > 0, d / np.where(se > 0, se, 1), 0))))
        w_sq = max(w_sq, dq / (1.0 + np.abs(ref_sq).max()))
    tag = "%s, lambda*=%g, alpha=%g" % (flow, lam, alpha)
    parity_report("50-step positions, " + tag, w_pos, 1e-3, "max |dr|")
    parity_report("50-step stress average, " + tag, w_se, 3.0, "max |dpi| / SE")
    parity_report("50-step stress second moment, " + tag, w_sq, 2e-2, "max |dq| / (1 + max|q|)")
    m.close()


def test_block_averaged_stress_config0(parity_report):
    # 2000 steps of the single 10^3 box under Lees-Edwards shear 0.1: block
    # averages over 100-step calls, GPU vs oracle within 3 combined SEs
    batch = S.single_shear_box(seed=1)
    m, op, boxes = _pair(batch, "lees_edwards", seed=1)
    L = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((1, 6), dtype=torch.float64, device="cuda")
    g_blocks, o_blocks = [], []
    for _ in range(20):
        m.advance(L, 100, st)
        g_blocks.append(st.cpu().numpy()[0].copy())
        ref, _, _ = O.advance(op, boxes[0], batch.L[0], 100)
        o_blocks.append(ref)
    m.sync()
    g = np.asarray(g_blocks)[2:]
    o = np.asarray(o_blocks)[2:]
    se = np.sqrt(g.var(axis=0, ddof=1) / len(g) + o.var(axis=0, ddof=1) / len(o))
    diff = np.abs(g.mean(axis=0) - o.mean(axis=0))
    assert np.all(diff <= 3 * se + 1e-6), (g.mean(0), o.mean(0), se)
    parity_report("2000-step block-averaged stress, 10^3 box, LE 0.1", float(np.max(diff / se)),
                  3.0, "max |dpi| / combined block SE")
    # eta_p = pi_xy / gdot and N1 = pi_xx - pi_yy are positive under shear
    assert g.mean(axis=0)[3] > 0
    m.close()


def test_checkpoint_resume_is_bitwise():
    # pair forces accumulate in fixed point (order-independent), so a step is
    # deterministic; the state (positions, velocities, forces, step) round-trips
    # exactly through get/set_state, and a resumed run repeats the continued one
    batch = _ragged_afbc_batch(seed=12)
    lh = _lh()
    gp = lh.dpd_params(flow="afbc", seed=4)
    m = lh.Micro.from_batch(gp, batch)
    L = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    m.advance(L, 10, st)
    ck = [m.get_state(b) for b in range(batch.n_boxes)]
    for b, (pos, vel, f, step, le) in enumerate(ck):
        m.set_state(b, pos, vel, f, step, le)
    again = [m.get_state(b) for b in range(batch.n_boxes)]
    for x, y in zip(ck, again):
        for u, v in zip(x[:3], y[:3]):
            assert np.array_equal(u, v)
        assert x[3] == y[3] == 10
    m.advance(L, 7, st)
    m.advance(L, 3, st)
    a = [m.get_state(b) for b in range(batch.n_boxes)]
    for b, (pos, vel, f, step, le) in enumerate(ck):
        m.set_state(b, pos, vel, f, step, le)
    m.advance(L, 10, st)
    bst = [m.get_state(b) for b in range(batch.n_boxes)]
    for x, y in zip(a, bst):
        assert x[3] == y[3] == 20
        for u, v in zip(x[:3], y[:3]):
            assert np.array_equal(u, v)
    m.close()


def test_subset_advance_touches_only_listed_boxes():
    batch = _ragged_afbc_batch(seed=2)
    lh = _lh()
    m = lh.Micro.from_batch(lh.dpd_params(flow="afbc", seed=2), batch)
    L = torch.from_numpy(batch.L).cuda()
    st = torch.full((batch.n_boxes, 6), 7.0, dtype=torch.float64, device="cuda")
    before = [m.get_state(b) for b in range(batch.n_boxes)]
    idx = torch.tensor([5, 1], dtype=torch.int32, device="cuda")
    m.advance(L, 4, st, box_idx_dev=idx)
    m.sync()
    out = st.cpu().numpy()
    for b in range(batch.n_boxes):
        after = m.get_state(b)
        if b in (1, 5):
            assert after[3] == 4 and not np.all(out[b] == 7.0)
        else:
            assert after[3] == 0 and np.array_equal(after[0], before[b][0])
            assert np.all(out[b] == 7.0)
    m.close()


def test_edge_cases_empty_and_minimal_boxes():
    lh = _lh()
    edges = np.array([3.0, 3.0, 4.0])
    n_beads = np.array([0, 81, 1], np.int32)
    L = np.zeros((3, 9), np.float32)
    b = S.make_batch(edges, L, 3, flow="afbc", n_beads=n_beads)
    b.n_chains = np.array([0, 4, 0], np.int32)
    m = lh.Micro.from_batch(lh.dpd_params(flow="afbc", seed=3), b)
    st = torch.zeros((3, 6), dtype=torch.float64, device="cuda")
    m.advance(torch.from_numpy(L).cuda(), 5, st)
    m.sync()
    out = st.cpu().numpy()
    assert np.all(out[0] == 0.0) and np.all(np.isfinite(out))
    # zero steps and an empty subset are no-ops
    m.advance(torch.from_numpy(L).cuda(), 0, st)
    m.advance(torch.from_numpy(L).cuda(), 3, st,
              box_idx_dev=torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert m.get_state(1)[3] == 5
    m.close()
    # an empty batch is valid
    e = lh.Micro(lh.dpd_params(), np.zeros((0, 3)), np.zeros(0, np.int32),
                 np.zeros(0, np.int32), 10, np.zeros((0, 3)), np.zeros((0, 3)))
    e.close()


def test_invalid_arguments_are_rejected():
    lh = _lh()
    with pytest.raises(lh.LhmmError) as ei:  # box narrower than 3 rc
        lh.Micro(lh.dpd_params(), np.array([[2.0, 5, 5]]), np.array([10], np.int32),
                 np.array([0], np.int32), 10, np.zeros((10, 3)), np.zeros((10, 3)))
    assert ei.value.status == lh.ERR_ARG
    with pytest.raises(lh.LhmmError) as ei:  # chains longer than the box
        lh.Micro(lh.dpd_params(), np.array([[5.0, 5, 5]]), np.array([10], np.int32),
                 np.array([2], np.int32), 10, np.zeros((10, 3)), np.zeros((10, 3)))
    assert ei.value.status == lh.ERR_ARG


def test_bond_overstretch_reported_without_fault():
    # host-side fault injection: a bond stretched past R0 is set as the state;
    # the kernel flags it, finishes the call and the host reads the status
    lh = _lh()
    batch = _ragged_afbc_batch(seed=1)
    m = lh.Micro.from_batch(lh.dpd_params(flow="afbc", seed=1), batch)
    pos, vel, f, step, le = m.get_state(3)
    pos = pos.copy()
    pos[1] = pos[0] + np.array([1.6, 0.0, 0.0])
    pos[1] = np.mod(pos[1], batch.edges[3])
    m.set_state(3, pos, vel, f, step, le)
    st = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    m.advance(torch.from_numpy(batch.L).cuda(), 1, st)
    status, per_box = m.sync(raise_on_error=False)
    assert status == lh.ERR_BOND_OVERSTRETCH
    assert per_box[3] & lh.BOX_BOND_OVERSTRETCH
    # the status is cleared by sync and the context stays usable
    assert m.sync(raise_on_error=False)[0] == lh.OK
    m.close()


def test_strong_extension_overstretches_on_both_sides():
    # planar extension through the overwritten BC shell pulls chains apart:
    # at rate 3 both the kernel and the oracle flag an over-stretched bond
    # within 100 steps, while the same boxes under rate-0.01 extension do not
    lh = _lh()
    edges = np.array([8.0, 9.0])
    for rate, expect in ((3.0, True), (0.01, False)):
        L = np.zeros((2, 9), np.float32)
        L[:, 0], L[:, 4] = rate, -rate
        batch = S.make_batch(edges, L, 31, flow="afbc")
        m, op, boxes = _pair(batch, "afbc", seed=31)
        st = torch.zeros((2, 6), dtype=torch.float64, device="cuda")
        m.advance(torch.from_numpy(batch.L).cuda(), 100, st)
        _, per_box = m.sync(raise_on_error=False)
        for b, ob in enumerate(boxes):
            _, _, err = O.advance(op, ob, batch.L[b], 100)
            gpu_flag = bool(per_box[b] & lh.BOX_BOND_OVERSTRETCH)
            orc_flag = bool(err & O.ERR_BOND_OVERSTRETCH)
            assert gpu_flag == orc_flag == expect, (rate, b, gpu_flag, orc_flag)
        m.close()


def test_host_buffer_entry_point_matches_device_one():
    batch = _ragged_afbc_batch(seed=6)
    lh = _lh()
    m1 = lh.Micro.from_batch(lh.dpd_params(flow="afbc", seed=6), batch)
    m2 = lh.Micro.from_batch(lh.dpd_params(flow="afbc", seed=6), batch)
    st = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    m1.advance(torch.from_numpy(batch.L).cuda(), 20, st)
    h = m2.advance_host(batch.L, 20)
    assert np.array_equal(st.cpu().numpy(), h)
    m1.close()
    m2.close()


def test_full_size_batch_sampled_parity():
    # the 1024-box workload in the launch configuration the benchmark times:
    # sampled boxes checked one by one against the oracle (initial forces and
    # the first step), and finite stresses everywhere after 100 steps
    batch = S.batched_microsolver()
    lh = _lh()
    m = lh.Micro.from_batch(lh.dpd_params(flow="afbc", seed=2), batch)
    op = O.dpd_params(flow_mode=O.FLOW_AFBC, seed=2)
    rng = np.random.default_rng(0)
    sample = list(rng.choice(batch.n_boxes, size=4, replace=False))
    sample.append(int(np.argmax(batch.n_beads)))
    oboxes = {}
    for b in sample:
        sl = batch.box_slice(b)
        ob = O.Box(batch.edges[b], batch.pos[sl], batch.vel[sl], int(batch.n_chains[b]),
                   batch.chain_len, box_id=b)
        O.compute_forces(op, ob, batch.L[b])
        oboxes[b] = ob
        assert np.abs(m.get_state(b)[2] - ob.force).max() <= 1e-4
    L = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    m.advance(L, 1, st)
    out = st.cpu().numpy()
    for b in sample:
        ref, _, _ = O.advance(op, oboxes[b], batch.L[b], 1)
        assert np.abs(out[b] - ref).max() <= 2e-3 * (1 + np.abs(ref).max()), (b, out[b], ref)
        assert np.abs(m.get_state(b)[2] - oboxes[b].force).max() <= 1e-4
    m.advance(L, 100, st)
    status, per_box = m.sync(raise_on_error=False)
    # boxes under the strongest planar extension may stretch a FENE bond to R0
    # under the literal AFBC overwrite (the oracle does too); that is reported,
    # never a non-finite state
    assert status in (lh.OK, lh.ERR_BOND_OVERSTRETCH)
    assert not np.any(per_box & lh.BOX_NAN)
    flagged = np.flatnonzero(per_box)
    assert np.all(batch.L[flagged, 4] != 0) and np.all(np.abs(batch.L[flagged, 0]) > 0.3)
    assert np.all(np.isfinite(st.cpu().numpy()))
    m.close()


def test_autotune_keeps_state_and_plan_is_valid():
    batch = _ragged_afbc_batch(seed=14)
    lh = _lh()
    m = lh.Micro.from_batch(lh.dpd_params(flow="afbc", seed=14), batch)
    L = torch.from_numpy(batch.L).cuda()
    before = [m.get_state(b) for b in range(batch.n_boxes)]
    m.autotune(L, probe_steps=3)
    after = [m.get_state(b) for b in range(batch.n_boxes)]
    for x, y in zip(before, after):
        for u, v in zip(x[:3], y[:3]):
            assert np.array_equal(u, v)
        assert x[3] == y[3] == 0
    plan = m.plan()
    assert sum(c["boxes"] for c in plan) == batch.n_boxes
    assert all(c["threads"] in (256, 512, 1024) for c in plan)
    # any variant gives the same physics to FP32 rounding: compare two plans
    m2 = lh.Micro.from_batch(lh.dpd_params(flow="afbc", seed=14), batch)
    for c in range(len(m2.plan())):
        m2.set_variant(c, 0)
    s1 = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    s2 = torch.zeros_like(s1)
    m.advance(L, 5, s1)
    m2.advance(L, 5, s2)
    m.sync()
    m2.sync()
    for b in range(batch.n_boxes):
        assert np.abs(m.get_state(b)[0] - m2.get_state(b)[0]).max() < 1e-4
    assert np.allclose(s1.cpu().numpy(), s2.cpu().numpy(), rtol=1e-3, atol=1e-3)
    m.close()
    m2.close()


def test_bonded_pairs_excluded_matches_oracle():
    # dpd_on_bonded = 0: no DPD pair force between chain neighbours
    batch = _ragged_afbc_batch(seed=6)
    m, op, boxes = _pair(batch, "afbc", seed=6, dpd_on_bonded=0)
    for b, ob in enumerate(boxes):
        _, _, f, _, _ = m.get_state(b)
        assert np.abs(f - ob.force).max() <= 1e-4, (b, np.abs(f - ob.force).max())
    m.close()


def test_afbc_peculiar_mode_matches_oracle(parity_report):
    # afbc_mode = 1: BC beads keep their velocity about their cell's BC mean;
    # the first step and, restarted from the GPU state, each later step's
    # update (beads whose region or cell the two precisions may choose
    # differently are left out and counted)
    from afbc_steps import ambiguous_beads, stepwise_afbc_parity
    batch = _ragged_afbc_batch(seed=21)
    m, op, boxes = _pair(batch, "afbc", seed=21, afbc_mode=1)
    L = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    m.advance(L, 1, st)
    m.sync()
    skipped = 0
    for b, ob in enumerate(boxes):
        O.advance(op, ob, batch.L[b], 1)
        _, vel, _, _, _ = m.get_state(b)
        amb = ambiguous_beads(ob.pos, batch.edges[b], 3, op.core_frac, op.bc_frac)
        ok = np.abs(vel - ob.vel).max(axis=1) <= 1e-4
        assert np.all(ok | amb), (b, np.abs(vel - ob.vel).max())
        skipped += int(np.count_nonzero(amb & ~ok))
    skipped += stepwise_afbc_parity(m, op, batch, 30)
    assert skipped <= 10
    parity_report("thermal-shell AFBC one-step map, 31 steps x 7 boxes, 3D", skipped, 10,
                  "bead velocities left out as ambiguous")
    m.close()


def test_issue_rate_probe_is_near_the_lane_count_times_clock():
    # bench.py's roofline denominator: SMs x 128 lanes x clock (<= ~2.07 GHz)
    import bench
    f, i = bench.issue_rate_probe(torch.cuda.current_stream().cuda_stream, iters=50)
    nominal = torch.cuda.get_device_properties(0).multi_processor_count * 128 * 2.07e9
    assert 0.3 * nominal < f < 1.05 * nominal, f
    assert 0.3 * nominal < i < 1.05 * nominal, i


@pytest.mark.parametrize("flow,afbc_mode", [("periodic", 0), ("afbc", 0), ("afbc", 1)])
def test_one_call_of_k_steps_equals_k_calls_of_one_step(flow, afbc_mode):
    # state carried across steps inside one launch must equal the state
    # carried through device memory between launches, bit for bit (a missing
    # barrier between the steps of one call would show here)
    lh = _lh()
    batch = _ragged_afbc_batch(seed=17)
    L = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    a = lh.Micro.from_batch(lh.dpd_params(flow=flow, seed=17, afbc_mode=afbc_mode), batch)
    b = lh.Micro.from_batch(lh.dpd_params(flow=flow, seed=17, afbc_mode=afbc_mode), batch)
    a.advance(L, 12, st)
    for _ in range(12):
        b.advance(L, 1, st)
    assert a.sync(raise_on_error=False)[0] == b.sync(raise_on_error=False)[0]
    for box in range(batch.n_boxes):
        for x, y in zip(a.get_state(box)[:4], b.get_state(box)[:4]):
            assert np.array_equal(np.asarray(x), np.asarray(y)), box
    a.close()
    b.close()


def test_full_advance_plan_chosen_by_autotune_gives_the_variants_results():
    # the autotuner may replace the size-class launches by one persistent
    # launch over every box (largest first) in one variant; a box's result
    # depends only on the variant that runs it, so a handle with every class
    # pinned to the chosen variants reproduces it bit for bit
    lh = _lh()
    batch = S.batched_microsolver(n_boxes=96, seed=23)
    L = torch.from_numpy(batch.L).cuda()
    a = lh.Micro.from_batch(lh.dpd_params(flow="afbc", seed=23), batch)
    b = lh.Micro.from_batch(lh.dpd_params(flow="afbc", seed=23), batch)
    a.autotune(L, probe_steps=3)
    plan = a.plan()
    variants = {(t, mb): k for k, (t, mb, gm) in enumerate(lh.MICRO_VARIANTS) if not gm}
    n_cls = len(b.plan())
    if len(plan) == 1 and n_cls > 1:  # one persistent launch
        for c in range(n_cls):
            b.set_variant(c, variants[(plan[0]["threads"], plan[0]["min_blocks"])])
    else:
        for c, p in enumerate(plan):
            b.set_variant(c, variants[(p["threads"], p["min_blocks"])])
    sa = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    sb = torch.zeros_like(sa)
    a.advance(L, 10, sa)
    b.advance(L, 10, sb)
    assert np.array_equal(sa.cpu().numpy(), sb.cpu().numpy())
    for box in (0, 17, 95):
        for x, y in zip(a.get_state(box)[:4], b.get_state(box)[:4]):
            assert np.array_equal(np.asarray(x), np.asarray(y))
    a.close()
    b.close()


@pytest.mark.parametrize("count", [0, 10, 152, 153, 200])
def test_device_list_advance_takes_each_listed_box_once(count):
    # the device-side count picks between the latency launch (up to one box
    # per SM) and the throughput launch (more boxes); either way every listed
    # box advances exactly once and moves as a host-listed subset advance
    # moves it (fixed-point pair forces: the launch shape does not change a
    # trajectory)
    lh = _lh()
    nb = 256
    edges = np.full(nb, 3.0)
    L = S.random_velocity_gradients(nb, 29, rate_range=(0.05, 0.5))
    batch = S.make_batch(edges, L, 29, flow="afbc")
    params = lh.dpd_params(flow="afbc", seed=29)
    a = lh.Micro.from_batch(params, batch)
    b = lh.Micro.from_batch(params, batch)
    perm = np.random.default_rng(29).permutation(nb).astype(np.int32)
    idx = torch.from_numpy(perm).cuda()
    cnt = torch.tensor([count], dtype=torch.int32, device="cuda")
    Lg = torch.from_numpy(batch.L).cuda()
    st_a = torch.zeros((nb, 6), dtype=torch.float64, device="cuda")
    st_b = torch.zeros_like(st_a)
    lh.check(lh.lib().lhmm_micro_advance_dev_count(a.h, lh._ptr(Lg), lh._ptr(idx), lh._ptr(cnt), nb,
                                                   7, lh._ptr(st_a), None, lh._stream_ptr(None)),
             "lhmm_micro_advance_dev_count")
    if count > 0:
        b.advance(Lg, 7, st_b, box_idx_dev=idx[:count].contiguous())
    assert a.sync(raise_on_error=False)[0] == b.sync(raise_on_error=False)[0] == lh.OK
    listed = set(perm[:count].tolist())
    for box in range(nb):
        pa, va, _, step_a, _ = a.get_state(box)
        pb, vb, _, step_b, _ = b.get_state(box)
        assert step_a == step_b == (7 if box in listed else 0), (box, step_a, step_b)
        assert np.array_equal(pa, pb) and np.array_equal(va, vb)
    a.close()
    b.close()


def test_list_variant_pins_and_errors():
    # a pinned list variant must hold the largest box; out-of-range indices
    # are argument errors; -1 restores the count-dependent default; every
    # shape moves the listed boxes identically
    lh = _lh()
    edges = np.array([13.0, 6.0, 8.0])  # 6 591 beads: no shared-memory plan holds the box
    L = S.random_velocity_gradients(3, 31, rate_range=(0.05, 0.5))
    batch = S.make_batch(edges, L, 31, flow="afbc")
    params = lh.dpd_params(flow="afbc", seed=31)
    m = lh.Micro.from_batch(params, batch)
    for bad in (-2, len(lh.MICRO_VARIANTS)):
        with pytest.raises(lh.LhmmError) as ei:
            m.set_list_variant(bad)
        assert ei.value.status == lh.ERR_ARG
    for v in (0, 2):  # shared-memory shapes cannot hold it
        with pytest.raises(lh.LhmmError) as ei:
            m.set_list_variant(v)
        assert ei.value.status == lh.ERR_UNSUPPORTED
    idx = torch.arange(3, dtype=torch.int32, device="cuda")
    Lg = torch.from_numpy(batch.L).cuda()
    states = []
    for v in (-1, 5, 6):  # default (device memory), 512 x 1 and 256 x 2 in device memory
        mm = lh.Micro.from_batch(params, batch)
        mm.set_list_variant(v)
        st = torch.zeros((3, 6), dtype=torch.float64, device="cuda")
        mm.advance(Lg, 6, st, box_idx_dev=idx)
        assert mm.sync(raise_on_error=False)[0] == lh.OK
        states.append([mm.get_state(b)[:2] for b in range(3)])
        mm.close()
    for other in states[1:]:
        for (pa, va), (pb, vb) in zip(states[0], other):
            assert np.array_equal(pa, pb) and np.array_equal(va, vb)
    m.close()
