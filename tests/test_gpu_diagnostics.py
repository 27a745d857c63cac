"""GPU FP64 momentum and energy diagnostics (lhmm_micro_diagnostics) against
the oracle's (Eq. motion's conserved quantities), through the C ABI."""
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


def _setup(flow, seed, L=None, **kw):
    from paper_2512_13267_gb300 import lhmm as lh
    edges = np.array([3.0, 5.0, 6.5, 8.0])
    if L is None:
        L = np.zeros((len(edges), 9), np.float32)
    batch = S.make_batch(edges, L, seed, flow=flow)
    fo = {"periodic": O.FLOW_PERIODIC, "lees_edwards": O.FLOW_LEES_EDWARDS,
          "afbc": O.FLOW_AFBC}[flow]
    m = lh.Micro.from_batch(lh.dpd_params(flow=flow, seed=seed, **kw), batch)
    op = O.dpd_params(flow_mode=fo, seed=seed, **kw)
    boxes = []
    for b in range(batch.n_boxes):
        sl = batch.box_slice(b)
        ob = O.Box(batch.edges[b], batch.pos[sl], batch.vel[sl], int(batch.n_chains[b]),
                   batch.chain_len, box_id=b)
        O.compute_forces(op, ob, batch.L[b])
        boxes.append(ob)
    return m, op, boxes, batch


def _diag(m, n):
    d = torch.zeros((n, 8), dtype=torch.float64, device="cuda")
    m.diagnostics(d)
    torch.cuda.synchronize()
    return d.cpu().numpy()


@pytest.mark.parametrize("flow,kw", [("periodic", {}), ("lees_edwards", {}),
                                     ("periodic", {"exclude_bonds": 2})])
def test_diagnostics_match_oracle_on_the_same_state(flow, kw, parity_report):
    L = None
    if flow == "lees_edwards":
        L = np.zeros((4, 9), np.float32)
        L[:, 1] = 0.5
    m, op, boxes, batch = _setup(flow, 7, L=L, **kw)
    st = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    m.advance(torch.from_numpy(batch.L).cuda(), 3, st)  # a nonzero Lees-Edwards offset
    m.sync()
    g = _diag(m, batch.n_boxes)
    worst = 0.0
    for b in range(batch.n_boxes):
        pos, vel, f, step, le = m.get_state(b)
        ob = O.Box(batch.edges[b], pos, vel, int(batch.n_chains[b]), batch.chain_len,
                   box_id=b, step=step, le_offset=le)
        ref, err = O.diagnostics(op, ob, batch.L[b])
        assert err == 0 and g[b, 7] == 0.0
        # same FP32 state on both sides: momentum and kinetic energy to FP64
        # rounding, potentials to the FP32 rounding of the pair distances
        assert np.abs(g[b, :3] - ref[:3]).max() <= 1e-9 * (1 + np.abs(vel).sum())
        assert abs(g[b, 3] - ref[3]) <= 1e-12 * ref[3]
        for k in (4, 5, 6):
            rel = abs(g[b, k] - ref[k]) / max(abs(ref[k]), 1.0)
            assert rel <= 2e-6, (b, k, g[b, k], ref[k])
            worst = max(worst, rel)
    parity_report("FP64 energy diagnostics, %s %s" % (flow, kw), worst, 2e-6,
                  "max relative |dU|")
    m.close()


def test_momentum_conserved_on_the_gpu_over_300_steps(parity_report):
    # periodic boxes at rest: pair forces are exact opposites (fixed-point sums)
    # and so are the bond forces, so the total momentum changes only by the
    # FP32 rounding of v += dt/2 F/m, a random walk of 2 x 300 half kicks over
    # N beads; the oracle keeps its P(0) to round-off
    m, op, boxes, batch = _setup("periodic", 11)
    n = batch.n_boxes
    p0 = _diag(m, n)[:, :3]
    st = torch.zeros((n, 6), dtype=torch.float64, device="cuda")
    m.advance(torch.from_numpy(batch.L).cuda(), 300, st)
    m.sync()
    g = _diag(m, n)
    for b in range(n):
        ref0, _ = O.diagnostics(op, boxes[b])
        O.advance(op, boxes[b], batch.L[b], 300)
        ref, _ = O.diagnostics(op, boxes[b])
        assert np.abs(ref[:3] - ref0[:3]).max() < 1e-10
        assert np.abs(p0[b] - ref0[:3]).max() < 1e-9 * (1 + batch.n_beads[b])
        vmax = max(np.abs(m.get_state(b)[1]).max(), 1.0)
        tol = 4.0 * np.sqrt(2 * 300 * batch.n_beads[b]) * 2.0 ** -24 * vmax
        drift = np.abs(g[b, :3] - p0[b]).max()
        assert drift <= tol, (b, drift, tol)
        parity_report("momentum drift over 300 steps, box %d" % b, drift, tol, "max |dP|")
        # 300 steps apart the FP32 and FP64 trajectories differ, but their
        # kinetic energies agree statistically (equipartition, 3 N kBT / 2)
        assert abs(g[b, 3] - ref[3]) <= 0.25 * ref[3]
    m.close()


def test_energy_after_fifty_steps_matches_oracle():
    m, op, boxes, batch = _setup("periodic", 13)
    st = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    m.advance(torch.from_numpy(batch.L).cuda(), 50, st)
    m.sync()
    g = _diag(m, batch.n_boxes)
    for b in range(batch.n_boxes):
        O.advance(op, boxes[b], batch.L[b], 50)
        ref, _ = O.diagnostics(op, boxes[b])
        for k in (3, 4, 5, 6):
            assert abs(g[b, k] - ref[k]) <= 2e-3 * max(abs(ref[k]), 1.0), (b, k, g[b, k], ref[k])
    m.close()
