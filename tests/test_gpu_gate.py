"""The surrogate gate inside the coupled macro step: closure inputs, the
all-DPD and all-surrogate limits, counters."""
import numpy as np
import pytest

from paper_2512_13267_gb300 import synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _system(seed=7, nx=8, ny=8, Ly=1.0):
    from paper_2512_13267_gb300 import lhmm as lh
    dh = Ly / ny
    Lx = nx * dh
    pos = S.sph_lattice(nx, ny, Lx, Ly, seed=seed, jitter=0.1).astype(np.float32)
    vel = np.random.default_rng(seed).normal(scale=0.05, size=pos.shape).astype(np.float32)
    n = pos.shape[0]
    batch = S.make_batch(np.full(n, 4.0), np.zeros((n, 9), np.float32), seed, flow="afbc")
    sp = lh.sph_params(n, 0, Lx=Lx, Ly=Ly, h=3 * dh, mass=dh * dh, rho0=1.0, c=2.0,
                       theta_pb=0.1, eta_s=0.2, dt=0.01, body_force=(0.3, 0.0),
                       body_mode=lh.SPH_BODY_REVERSE_POISEUILLE)
    sph = lh.Sph(sp, pos, vel)
    micro = lh.Micro.from_batch(lh.dpd_params(flow="afbc", seed=5, alpha=0.05), batch)
    cpl = lh.Coupled(sph, micro, 4, 6)
    cpl.micro_batch, cpl.micro_params, cpl.k_micro = batch, lh.dpd_params(
        flow="afbc", seed=5, alpha=0.05), 6
    clo = lh.Closure(members=5, in_dim=67, hidden=256, n_hidden=4, out_dim=3, seed=2)
    clo.set_normalization(np.zeros(67), np.ones(67), np.full(3, 1e-3))
    return cpl, clo


def test_closure_inputs_hold_gradient_history_and_stress():
    cpl, clo = _system()
    cpl.set_closure(clo, threshold=0.02)
    Ls, Ss = [], []
    for _ in range(18):
        _, st_before = cpl.exchange()
        cpl.step(1, use_graph=True)
        L, _ = cpl.exchange()
        Ls.append(L[:, [0, 1, 3, 4]].copy())
        Ss.append(st_before[:, [0, 3, 1]].astype(np.float32))
    X = cpl.closure_inputs()
    hist = np.stack(Ls[-16:], axis=1).reshape(X.shape[0], 64)
    assert np.array_equal(X[:, :64], hist)
    assert np.array_equal(X[:, 64:67], Ss[-1])


def test_zero_threshold_gate_equals_plain_step():
    # the gated step's DPD boxes run in the list launch; pinned to the
    # variant of the plain step's class plan (these 192-bead boxes start at
    # 256 threads x 4 blocks, variant 0) it reproduces the plain step bit
    # for bit, stresses included
    a, ca = _system(seed=9)
    b, cb = _system(seed=9)
    assert [(p["threads"], p["min_blocks"]) for p in a.micro.plan()] == [(256, 4)]
    b.micro.set_list_variant(0)
    a.set_closure(ca, threshold=0.0)
    b.set_closure(cb, threshold=0.0)
    a.step(3, use_graph=True)
    b.step(3, use_graph=True)
    b.enable_gate(True)
    a.step(3, use_graph=True)
    b.step(3, use_graph=True)  # eager, capture, replay of the gated graph
    La, sa = a.exchange()
    Lb, sb = b.exchange()
    assert np.array_equal(La, Lb) and np.array_equal(sa, sb)
    st = b.gate_stats()
    assert st["gated_steps"] == 3 and st["dpd_boxes"] == 3 * b.n_boxes


def test_default_list_variant_gives_the_plain_step_to_summation_order():
    # with its default (latency-first) variant the list launch moves every
    # bead exactly as the class plan does: the fixed-point pair forces do
    # not depend on the launch shape; the FP32 virial sums may differ in the
    # last bits, so the coupled fields after three gated steps agree to
    # rounding
    a, ca = _system(seed=9)
    b, cb = _system(seed=9)
    a.set_closure(ca, threshold=0.0)
    b.set_closure(cb, threshold=0.0)
    a.step(3, use_graph=True)
    b.step(3, use_graph=True)
    b.enable_gate(True)
    a.step(1, use_graph=False)
    b.step(1, use_graph=False)
    pa = [a.micro.get_state(k)[0] for k in range(a.n_boxes)]
    pb = [b.micro.get_state(k)[0] for k in range(b.n_boxes)]
    assert all(np.array_equal(x, y) for x, y in zip(pa, pb))
    a.step(2, use_graph=True)
    b.step(2, use_graph=True)
    La, sa = a.exchange()
    Lb, sb = b.exchange()
    assert np.allclose(La, Lb, rtol=1e-4, atol=1e-6) and np.allclose(sa, sb, rtol=1e-4, atol=1e-9)


def test_open_gate_freezes_boxes_and_applies_prediction():
    cpl, clo = _system(seed=11)
    cpl.set_closure(clo, threshold=1e30, audit_every=0)
    cpl.step(17, use_graph=True)
    steps_before = [cpl.micro.get_state(b)[3] for b in range(cpl.n_boxes)]
    _, st0 = cpl.exchange()
    cpl.enable_gate(True)
    cpl.step(1, use_graph=False)
    X = cpl.closure_inputs()
    _, st1 = cpl.exchange()
    assert [cpl.micro.get_state(b)[3] for b in range(cpl.n_boxes)] == steps_before
    mean = torch.zeros((cpl.n_boxes, 3), dtype=torch.float32, device="cuda")
    spread = torch.zeros(cpl.n_boxes, dtype=torch.float32, device="cuda")
    clo.infer(torch.from_numpy(X).cuda(), mean, spread)
    d = st1[:, [0, 3, 1]] - st0[:, [0, 3, 1]]
    assert np.allclose(d, mean.cpu().numpy(), rtol=1e-5, atol=1e-7)
    assert np.array_equal(st1[:, [2, 4, 5]], st0[:, [2, 4, 5]])
    assert cpl.gate_stats()["dpd_boxes"] == 0


def test_audit_share_runs_dpd_and_measures_error():
    cpl, clo = _system(seed=13)
    cpl.set_closure(clo, threshold=1e30, audit_every=4)
    cpl.step(17, use_graph=True)
    cpl.enable_gate(True)
    cpl.step(4, use_graph=True)
    st = cpl.gate_stats()
    assert st["gated_steps"] == 4
    assert st["dpd_boxes"] == st["audited"] == 4 * cpl.n_boxes // 4
    assert st["audit_ref2"] > 0 and st["audit_err2"] > 0


def test_set_gate_keeps_history_and_switches_threshold():
    cpl, clo = _system(seed=15)
    cpl.set_closure(clo, threshold=1e30, audit_every=0)
    cpl.step(17, use_graph=True)
    X0 = cpl.closure_inputs()
    cpl.set_gate(0.0, 0)
    assert np.array_equal(cpl.closure_inputs(), X0)
    cpl.enable_gate(True)
    cpl.step(2, use_graph=True)
    st = cpl.gate_stats()
    assert st["gated_steps"] == 2 and st["dpd_boxes"] == 2 * cpl.n_boxes
    cpl.set_gate(1e30, 0)
    cpl.step(3, use_graph=True)  # eager, capture, replay with the new threshold
    st2 = cpl.gate_stats()
    assert st2["gated_steps"] == 5 and st2["dpd_boxes"] == st["dpd_boxes"]


def test_absolute_mode_sets_stress_to_prediction():
    cpl, clo = _system(seed=17)
    cpl.set_closure(clo, threshold=1e30, audit_every=0)
    cpl.set_gate(1e30, 0, absolute=True)
    cpl.step(17, use_graph=True)
    assert np.all(cpl.closure_inputs()[:, 64:67] == 0.0)
    _, st0 = cpl.exchange()
    cpl.enable_gate(True)
    cpl.step(1, use_graph=False)
    X = cpl.closure_inputs()
    assert np.all(X[:, 64:67] == 0.0)
    _, st1 = cpl.exchange()
    mean = torch.zeros((cpl.n_boxes, 3), dtype=torch.float32, device="cuda")
    spread = torch.zeros(cpl.n_boxes, dtype=torch.float32, device="cuda")
    clo.infer(torch.from_numpy(X).cuda(), mean, spread)
    assert np.allclose(st1[:, [0, 3, 1]], mean.cpu().numpy(), rtol=1e-6, atol=1e-9)
    assert np.array_equal(st1[:, [2, 4, 5]], st0[:, [2, 4, 5]])
    assert cpl.gate_stats()["dpd_boxes"] == 0


@pytest.mark.parametrize("warm,expect_extra", [(-1, 6), (0, 0), (3, 3)])
def test_frozen_boxes_warm_up_when_they_return(warm, expect_extra):
    # boxes frozen by the gate run `warm` discarded DPD steps (-1: k' = 6)
    # before their sampled k' steps when the gate sends them back to DPD
    cpl, clo = _system(seed=19)
    cpl.set_closure(clo, threshold=1e30, audit_every=0)
    cpl.step(17, use_graph=True)
    cpl.enable_gate(True)
    cpl.step(1, use_graph=False)          # every box trusted: all frozen
    before = [cpl.micro.get_state(b)[3] for b in range(cpl.n_boxes)]
    cpl.set_gate(0.0, 0, warmup_steps=warm)  # now every box runs DPD
    cpl.step(1, use_graph=False)
    after = [cpl.micro.get_state(b)[3] for b in range(cpl.n_boxes)]
    assert all(a - b == 6 + expect_extra for a, b in zip(after, before))
    cpl.step(1, use_graph=False)          # no box was frozen in between: no warm-up
    again = [cpl.micro.get_state(b)[3] for b in range(cpl.n_boxes)]
    assert all(a - b == 6 for a, b in zip(again, after))


def test_onpolicy_labels_are_the_dpd_stress_when_every_box_runs_dpd():
    # with a zero threshold every box runs DPD in the gated step, so the
    # shadow batch (cloned state, same gradients) must give the same stress
    from paper_2512_13267_gb300 import closure
    from paper_2512_13267_gb300 import lhmm as lh
    cpl, clo = _system(seed=11)
    cpl.set_closure(clo, threshold=0.0)
    cpl.step(2, use_graph=True)
    cpl.enable_gate(True)
    shadow = lh.Micro.from_batch(cpl.micro_params, cpl.micro_batch)
    X, T = closure.onpolicy_pairs(cpl, shadow, 3, absolute=True)
    n = cpl.n_boxes
    assert X.shape == (3 * n, 67) and T.shape == (3 * n, 3)
    _, st = cpl.exchange()
    ref = st[:, [0, 3, 1]]
    assert np.abs(T[-n:] - ref).max() <= 1e-5 * (1.0 + np.abs(ref).max())
    for o in (shadow, cpl, clo):
        o.close()


def test_large_mixed_run_small_cylinder_cell_gated_step():
    # the large mixed run's pipeline (cylinder array with wall particles, one
    # box per fluid particle, autotuned launches, pairs, training, gated
    # graph-replayed macro steps) at a small size: it runs, the walls carry
    # no box, the device reports no fault and the gated share is a fraction
    from paper_2512_13267_gb300 import closure
    out = closure.large_mixed_run(n_fluid=256, cell=4.0, box_beads=375, warm=2, n_data=20,
                                  train_steps=40, timing_steps=3, threshold=0.02, audit_every=5)
    assert out["device_status"] == "ok"
    assert out["macro_steps_per_s_plain"] > 0 and out["macro_steps_per_s_surrogate"] > 0
    assert 0.0 <= out["dpd_fraction"] <= 1.0
    assert "wall SPH" in out["workload"] and out["train_pairs"] > 0


def test_online_calibration_fits_the_audits():
    # every trusted box audited (audit_every = 1): all boxes run DPD, so two
    # systems whose closures differ only by a shifted output bias (every
    # member's prediction moved by delta, the ensemble spread unchanged) see
    # the same flow, and the fitted lines must be a' = a, c' = c - a delta
    # (whatever a is, also where it is held at a bound); with the calibration
    # off the map stays the identity
    delta_n, out_scale = 2.0, 1e-3  # shift in normalised output units; _system's output scale
    systems = []
    for shift in (False, True):
        cpl, clo = _system(seed=19)
        if shift:
            for m in range(5):
                p = clo.get_params(m)
                p[-3:] += delta_n  # b of the output layer
                clo.set_params(m, p)
        cpl.set_closure(clo, threshold=1e30, audit_every=1)
        cpl.step(17, use_graph=True)
        cpl.set_online_calibration(True, decay=0.8)
        cpl.enable_gate(True)
        cpl.step(5, use_graph=True)
        systems.append((cpl, clo))
    (a, _), (b, _) = systems
    La, sa = a.exchange()
    Lb, sb = b.exchange()
    assert np.array_equal(La, Lb) and np.array_equal(sa, sb)
    ma = a.set_online_calibration(-1)
    mb = b.set_online_calibration(-1)
    assert not np.allclose(ma, [[1, 0], [1, 0], [1, 0]])
    assert np.allclose(mb[:, 0], ma[:, 0], rtol=1e-4), (ma, mb)
    shift = ma[:, 0] * delta_n * out_scale
    assert np.allclose(mb[:, 1], ma[:, 1] - shift, rtol=0, atol=1e-3 * np.abs(shift).max()), (ma, mb)
    c, cc = _system(seed=19)
    c.set_closure(cc, threshold=1e30, audit_every=1)
    c.step(17, use_graph=True)
    c.enable_gate(True)
    c.step(3, use_graph=True)
    assert np.array_equal(c.set_online_calibration(-1), [[1, 0], [1, 0], [1, 0]])
