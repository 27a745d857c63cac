"""Boxes held in device memory (kernel variants 5 and 6) instead of one SM's
shared memory: bit-identical to the shared-memory variant with the same
threads per block, and parity with the FP64 oracle for boxes too large for
shared memory (up to the paper's 76 x 76 melt box, Table 2)."""
import numpy as np
import pytest

import oracle as O
from paper_2512_13267_gb300 import synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PAPER_2D = dict(a_ij=25.0, gamma=4.5, sigma=3.0, H_fene=50.0, R0=1.5, dt=0.005)
FLOW_O = {"periodic": O.FLOW_PERIODIC, "lees_edwards": O.FLOW_LEES_EDWARDS, "afbc": O.FLOW_AFBC}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _lh():
    from paper_2512_13267_gb300 import lhmm
    return lhmm


def _batch3d(flow, seed):
    edges = np.array([3.0, 5.0, 6.0, 7.5, 9.0, 12.0])
    if flow == "lees_edwards":
        L = np.zeros((len(edges), 9), np.float32)
        L[:, 1] = np.linspace(0.05, 0.5, len(edges))
    else:
        L = S.random_velocity_gradients(len(edges), seed, rate_range=(0.05, 1.0))
    return S.make_batch(edges, L, seed, flow=flow)


def _run(batch, params, variant, steps):
    lh = _lh()
    m = lh.Micro.from_batch(params, batch)
    for c in range(len(m.plan())):
        m.set_variant(c, variant)
    L = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    sq = torch.zeros_like(st)
    m.advance(L, steps, st, sq)
    status = m.sync(raise_on_error=False)[0]
    states = [m.get_state(b) for b in range(batch.n_boxes)]
    m.close()
    return st.cpu().numpy(), sq.cpu().numpy(), states, status


@pytest.mark.parametrize("flow,afbc_mode,dim", [("periodic", 0, 3), ("lees_edwards", 0, 3),
                                                ("afbc", 0, 3), ("afbc", 1, 3), ("afbc", 0, 2)])
@pytest.mark.parametrize("smem_v,gm_v", [(4, 5), (3, 6)])
def test_device_memory_variant_is_bitwise_equal_to_shared(flow, afbc_mode, dim, smem_v, gm_v):
    lh = _lh()
    assert lh.MICRO_VARIANTS[smem_v][:2] == lh.MICRO_VARIANTS[gm_v][:2]
    assert not lh.MICRO_VARIANTS[smem_v][2] and lh.MICRO_VARIANTS[gm_v][2]
    if dim == 2:
        edges = np.array([3.0, 8.0, 12.0, 20.0])
        L = np.zeros((4, 9), np.float32)
        L[:, 1] = 0.1
        n = np.rint(4 * edges * edges).astype(int)
        n -= n % 8
        batch = S.make_batch(edges, L, 5, flow=flow, chain_len=8, fraction=1.0, n_beads=n, dim=2)
        params = lh.dpd_params(flow=flow, seed=5, dim=2, afbc_mode=afbc_mode, **PAPER_2D)
    else:
        batch = _batch3d(flow, 5)
        params = lh.dpd_params(flow=flow, seed=5, afbc_mode=afbc_mode)
    a = _run(batch, params, smem_v, 30)
    b = _run(batch, params, gm_v, 30)
    assert a[3] == b[3]
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for sa, sb in zip(a[2], b[2]):
        for x, y in zip(sa, sb):
            assert np.array_equal(np.asarray(x), np.asarray(y))


def _oracle_boxes(batch, op):
    boxes = []
    for b in range(batch.n_boxes):
        sl = batch.box_slice(b)
        ob = O.Box(batch.edges[b], batch.pos[sl], batch.vel[sl], int(batch.n_chains[b]),
                   batch.chain_len, box_id=b)
        O.compute_forces(op, ob, batch.L[b])
        boxes.append(ob)
    return boxes


def _minimage(d, E):
    return d - E * np.rint(d / E)


@pytest.mark.parametrize("flow", ["periodic", "afbc"])
def test_3d_box_beyond_shared_memory_matches_oracle(flow):
    # 14^3 box at density 3: 8232 beads, more than one SM's shared memory holds
    lh = _lh()
    edges = np.array([14.0, 6.0])
    L = S.random_velocity_gradients(2, 7, rate_range=(0.1, 0.5))
    batch = S.make_batch(edges, L, 7, flow=flow)
    assert batch.n_beads[0] > 5700
    m = lh.Micro.from_batch(lh.dpd_params(flow=flow, seed=7), batch)
    op = O.dpd_params(flow_mode=FLOW_O[flow], seed=7)
    boxes = _oracle_boxes(batch, op)
    plan = m.plan()
    assert any(c["max_beads"] == batch.n_beads[0] for c in plan)
    for b, ob in enumerate(boxes):
        _, _, f, _, _ = m.get_state(b)
        assert np.abs(f - ob.force).max() <= 1e-4, (b, np.abs(f - ob.force).max())
    Lg = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((2, 6), dtype=torch.float64, device="cuda")
    m.advance(Lg, 20, st)
    assert m.sync(raise_on_error=False)[0] == lh.OK
    got = st.cpu().numpy()
    for b, ob in enumerate(boxes):
        ref, _, err = O.advance(op, ob, batch.L[b], 20)
        assert err == 0
        pos, _, _, step, _ = m.get_state(b)
        assert step == 20
        assert np.abs(_minimage(pos - ob.pos, batch.edges[b][0])).max() <= 1e-3
        scale = 1.0 + np.abs(ref).max()
        assert np.abs(got[b] - ref).max() <= 2e-2 * scale, (b, got[b], ref)
    m.close()


def test_paper_76x76_melt_box_matches_oracle():
    # the paper's micro-domain (Table 2): a 76 x 76 2D melt of N_d = 8 chains
    # at number density 4 (23 104 beads) under planar shear through the AFBC
    # shell; it runs in the device-memory variant
    lh = _lh()
    edges = np.array([76.0])
    L = np.zeros((1, 9), np.float32)
    L[0, 1] = 0.01
    n = np.array([4 * 76 * 76])
    batch = S.make_batch(edges, L, 9, flow="afbc", chain_len=8, fraction=1.0, n_beads=n, dim=2)
    params = lh.dpd_params(flow="afbc", seed=9, dim=2, **PAPER_2D)
    m = lh.Micro.from_batch(params, batch)
    assert m.info()[2] == 23104
    op = O.dpd_params(flow_mode=O.FLOW_AFBC, seed=9, dim=2, **PAPER_2D)
    (ob,) = _oracle_boxes(batch, op)
    _, _, f, _, _ = m.get_state(0)
    assert np.abs(f - ob.force).max() <= 1e-4
    Lg = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((1, 6), dtype=torch.float64, device="cuda")
    m.advance(Lg, 10, st)
    assert m.sync(raise_on_error=False)[0] == lh.OK
    ref, _, err = O.advance(op, ob, batch.L[0], 10)
    assert err == 0
    pos, vel, _, _, _ = m.get_state(0)
    assert np.all(vel[:, 2] == 0.0)
    assert np.abs(_minimage(pos - ob.pos, 76.0)).max() <= 1e-3
    got = st.cpu().numpy()[0]
    assert np.abs(got - ref).max() <= 2e-2 * (1.0 + np.abs(ref).max()), (got, ref)
    m.close()


@pytest.mark.parametrize("afbc_mode", [0, 1])
def test_device_list_advance_of_large_boxes_equals_plain_advance(afbc_mode):
    # the persistent launch over a device-side box list (what a gated
    # coupled step uses) in the device-memory variant: same states and
    # stresses as the per-class launch, bit for bit
    lh = _lh()
    edges = np.array([40.0, 44.0, 42.0])
    L = np.zeros((3, 9), np.float32)
    L[:, 1] = [0.02, 0.05, 0.1]
    n = np.rint(4 * edges * edges).astype(int)
    n -= n % 8
    batch = S.make_batch(edges, L, 13, flow="afbc", chain_len=8, fraction=1.0, n_beads=n, dim=2)
    assert batch.n_beads.min() > 5700
    params = lh.dpd_params(flow="afbc", seed=13, dim=2, afbc_mode=afbc_mode, **PAPER_2D)
    a = lh.Micro.from_batch(params, batch)
    b = lh.Micro.from_batch(params, batch)
    Lg = torch.from_numpy(batch.L).cuda()
    st_a = torch.zeros((3, 6), dtype=torch.float64, device="cuda")
    st_b = torch.zeros_like(st_a)
    a.advance(Lg, 20, st_a)
    idx = torch.arange(3, dtype=torch.int32, device="cuda")
    cnt = torch.tensor([3], dtype=torch.int32, device="cuda")
    lh.check(lh.lib().lhmm_micro_advance_dev_count(b.h, lh._ptr(Lg), lh._ptr(idx), lh._ptr(cnt), 3,
                                                   20, lh._ptr(st_b), None, lh._stream_ptr(None)),
             "lhmm_micro_advance_dev_count")
    assert a.sync(raise_on_error=False)[0] == b.sync(raise_on_error=False)[0] == lh.OK
    assert torch.equal(st_a, st_b)
    for box in range(3):
        for x, y in zip(a.get_state(box)[:4], b.get_state(box)[:4]):
            assert np.array_equal(np.asarray(x), np.asarray(y))
    a.close()
    b.close()


@pytest.mark.parametrize("dim,edge,n", [(3, 27.0, 3 * 27 ** 3), (2, 127.0, 64512)])
def test_largest_supported_boxes_match_oracle(dim, edge, n):
    # the size limits of the engine (16-bit bead and cell ids): a 27^3 box of
    # 59 049 beads and 19 683 cells, and a 127 x 127 2D melt of 64 512 beads
    # (16 129 cells), both under a velocity gradient through the AFBC shell
    lh = _lh()
    L = np.zeros((1, 9), np.float32)
    L[0, 1] = 0.05
    if dim == 3:
        batch = S.make_batch(np.array([edge]), L, 11, flow="afbc", n_beads=np.array([n]))
        params = lh.dpd_params(flow="afbc", seed=11)
        op = O.dpd_params(flow_mode=O.FLOW_AFBC, seed=11)
    else:
        batch = S.make_batch(np.array([edge]), L, 11, flow="afbc", chain_len=8, fraction=1.0,
                             n_beads=np.array([n]), dim=2)
        params = lh.dpd_params(flow="afbc", seed=11, dim=2, **PAPER_2D)
        op = O.dpd_params(flow_mode=O.FLOW_AFBC, seed=11, dim=2, **PAPER_2D)
    assert batch.n_beads[0] == n <= 65535
    m = lh.Micro.from_batch(params, batch)
    (ob,) = _oracle_boxes(batch, op)
    _, _, f, _, _ = m.get_state(0)
    assert np.abs(f - ob.force).max() <= 1e-4
    Lg = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((1, 6), dtype=torch.float64, device="cuda")
    m.advance(Lg, 5, st)
    assert m.sync(raise_on_error=False)[0] == lh.OK
    ref, _, err = O.advance(op, ob, batch.L[0], 5)
    assert err == 0
    pos, _, _, step, _ = m.get_state(0)
    assert step == 5
    assert np.abs(_minimage(pos - ob.pos, edge)).max() <= 1e-3
    got = st.cpu().numpy()[0]
    assert np.abs(got - ref).max() <= 2e-2 * (1.0 + np.abs(ref).max()), (got, ref)
    m.close()


def test_boxes_past_the_id_limits_are_rejected_on_the_host():
    # 65 536 beads, or more than 65 535 cells, do not fit the 16-bit ids: the
    # handle is refused before anything runs on the device
    lh = _lh()
    n = 65536
    with pytest.raises(lh.LhmmError) as ei:
        lh.Micro(lh.dpd_params(), np.array([[28.0, 28.0, 28.0]]), np.array([n], np.int32),
                 np.array([0], np.int32), 10, np.zeros((n, 3)), np.zeros((n, 3)))
    assert ei.value.status == lh.ERR_ARG
    n = 1000  # sparse box of 41^3 = 68 921 cells
    with pytest.raises(lh.LhmmError) as ei:
        lh.Micro(lh.dpd_params(), np.array([[41.0, 41.0, 41.0]]), np.array([n], np.int32),
                 np.array([0], np.int32), 10, np.random.default_rng(0).uniform(0, 41, (n, 3)),
                 np.zeros((n, 3)))
    assert ei.value.status == lh.ERR_UNSUPPORTED
    # a Lees-Edwards row stores the x cell offset of its sliding image in
    # 8 bits: more than 60 cells along x is refused as well
    n = 400
    with pytest.raises(lh.LhmmError) as ei:
        lh.Micro(lh.dpd_params(flow="lees_edwards", dim=2), np.array([[61.0, 10.0, 1.0]]),
                 np.array([n], np.int32), np.array([0], np.int32), 10,
                 np.random.default_rng(1).uniform(0, 10, (n, 3)) * [6.1, 1.0, 0.0],
                 np.zeros((n, 3)))
    assert ei.value.status == lh.ERR_UNSUPPORTED
