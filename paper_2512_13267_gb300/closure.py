"""Learned-closure workflow over the C ABI: collect (input, stress increment)
pairs from plain coupled macro steps, normalise, train the ensemble on the
GPU, and compare a surrogate-gated run with a plain one.

The closure is not part of the paper; it is this library's surrogate layer.
Inputs: the 16 past velocity gradients (Lxx, Lxy, Lyx, Lyy) of a particle,
oldest first, and its current polymer stress (pi_xx, pi_xy, pi_yy); target:
the increment of (pi_xx, pi_xy, pi_yy) over one macro step.
"""
import time

import numpy as np

from . import lhmm

N_IN = 67
N_OUT = 3
HIST = 16
STRESS_COLS = [0, 3, 1]  # xx, xy, yy in the micro stress layout


def collect_pairs(coupled, n_steps, skip=HIST, absolute=False):
    """Run n_steps plain macro steps (gate off, closure attached) and return
    inputs X (m x 67) and targets T (m x 3): the increment of (pi_xx, pi_xy,
    pi_yy) over the step, or with `absolute` the stress after it (the gate
    must be in its absolute mode, so that the stress inputs are zero); the
    first `skip` steps only fill the gradient history."""
    coupled.enable_gate(False)
    Xs, Ts = [], []
    for k in range(n_steps):
        coupled.step(1, use_graph=True)
        if k < skip:
            continue
        X = coupled.closure_inputs()
        _, st = coupled.exchange()
        T = st[:, STRESS_COLS].astype(np.float32)
        if not absolute:
            T = T - X[:, 64:67]
        Xs.append(X)
        Ts.append(T)
    if not Xs:
        return np.zeros((0, N_IN), np.float32), np.zeros((0, N_OUT), np.float32)
    return np.concatenate(Xs), np.concatenate(Ts)


def normalization(X, T, floor=1e-6):
    mean = X.mean(axis=0)
    std = np.maximum(X.std(axis=0), floor)
    scale = np.maximum(T.std(axis=0), floor)
    return mean.astype(np.float32), std.astype(np.float32), scale.astype(np.float32)


def train(closure, X, T, steps, batch=4096, lr=1e-3, weight_decay=1e-4, seed=0, log_every=0,
          cosine=False):
    """AdamW on bootstrap batches (each member draws its own rows), learning
    rate lr with cosine decay to zero over `steps` (cosine=True).  Returns the
    per-member loss history (every log_every steps) and the wall time."""
    import torch
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    batch = max(32, min(batch, (n // 32) * 32))
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    Td = torch.from_numpy(np.ascontiguousarray(T, np.float32)).cuda()
    loss = torch.zeros(closure.members, dtype=torch.float32, device="cuda")
    rows_all = torch.from_numpy(
        rng.integers(0, n, size=(min(steps, 64), closure.members, batch)).astype(np.int32)).cuda()
    hist = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        rows = rows_all[k % rows_all.shape[0]]
        if k % rows_all.shape[0] == 0 and k > 0:
            rows_all = torch.randint(0, n, rows_all.shape, dtype=torch.int32, device="cuda")
        lr_k = lr * 0.5 * (1.0 + np.cos(np.pi * k / steps)) if cosine else lr
        closure.train_step(Xd, Td, batch, lr_k, weight_decay, rows_dev=rows, loss_dev=loss)
        if log_every and (k % log_every == 0 or k == steps - 1):
            hist.append(loss.cpu().numpy().copy())
    torch.cuda.synchronize()
    return hist, time.perf_counter() - t0


def calibrate(closure, X_val, T_val, out_scale):
    """Per-output linear recalibration of the ensemble mean on held-out pairs:
    fit T ~ a * prediction + c by least squares and fold (a, c) into every
    member's output layer (W_out row k times a_k, b_out[k] -> a_k b_out[k] +
    c_k / out_scale_k).  Returns (a, c)."""
    import torch
    Xd = torch.from_numpy(np.ascontiguousarray(X_val, np.float32)).cuda()
    Y = closure.forward_members(Xd).mean(axis=0) * np.asarray(out_scale)[None, :]
    a = np.ones(closure.out_dim)
    c = np.zeros(closure.out_dim)
    for k in range(closure.out_dim):
        A = np.stack([Y[:, k], np.ones(len(Y))], axis=1).astype(np.float64)
        sol, *_ = np.linalg.lstsq(A, T_val[:, k].astype(np.float64), rcond=None)
        a[k], c[k] = sol
    d_hidden = closure.dims[-2]
    for m in range(closure.members):
        prm = closure.get_params(m).astype(np.float64)
        b0 = prm.size - closure.out_dim
        w0 = b0 - closure.out_dim * d_hidden
        W = prm[w0:b0].reshape(closure.out_dim, d_hidden)
        b = prm[b0:]
        W *= a[:, None]
        prm[w0:b0] = W.ravel()
        prm[b0:] = a * b + c / np.asarray(out_scale, np.float64)
        closure.set_params(m, prm.astype(np.float32))
    return a, c


def binned_profiles(y, stress6, Ly, nbins=16):
    """y-binned pi_xy and N1 = pi_xx - pi_yy of the fluid particles."""
    k = np.minimum((np.asarray(y) / Ly * nbins).astype(int), nbins - 1)
    cnt = np.maximum(np.bincount(k, minlength=nbins), 1)
    pxy = np.bincount(k, weights=stress6[:, 3], minlength=nbins) / cnt
    n1 = np.bincount(k, weights=stress6[:, 0] - stress6[:, 1], minlength=nbins) / cnt
    return pxy, n1


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _channel(seed, alpha, U_o, c_factor, eta_s, k_micro, dt_dpd, members, closure_seed):
    from . import synth
    sph_cfg, batch = synth.coupled_channel(seed=seed, U_o=U_o, c_factor=c_factor, eta_s=eta_s,
                                           delta_t=k_micro * dt_dpd)
    M = sph_cfg["substeps"]
    sp = lhmm.sph_params(sph_cfg["pos"].shape[0], 0, Lx=sph_cfg["Lx"], Ly=sph_cfg["Ly"],
                         h=sph_cfg["h"], mass=sph_cfg["mass"], rho0=1.0, c=sph_cfg["c"],
                         theta_pb=0.1, eta_s=eta_s, dt=sph_cfg["dt"],
                         body_force=(sph_cfg["body_force"], 0.0),
                         body_mode=lhmm.SPH_BODY_REVERSE_POISEUILLE)
    sph = lhmm.Sph(sp, sph_cfg["pos"], sph_cfg["vel"])
    params = lhmm.dpd_params(flow="afbc", seed=seed, alpha=alpha)
    micro = lhmm.Micro.from_batch(params, batch)
    cpl = lhmm.Coupled(sph, micro, M, k_micro)
    cpl.micro_batch, cpl.micro_params, cpl.k_micro = batch, params, k_micro
    clo = lhmm.Closure(members=members, in_dim=N_IN, hidden=256, n_hidden=4, out_dim=N_OUT,
                       seed=closure_seed)
    return cpl, clo, sph_cfg, M


def onpolicy_pairs(gated, shadow, n_steps, absolute=False, lockstep=()):
    """Training pairs from the flow the gated system actually produces
    (dataset aggregation): `shadow` is a micro batch holding the same boxes,
    started from the gated system's micro state, that runs DPD for every
    particle under the gradients the gated macro step exports.  Its stress is
    the label the closure should have given each particle in that flow,
    including the trusted ones.  Systems in `lockstep` take one plain step per
    gated step."""
    import torch
    nb = gated.n_boxes
    for b in range(nb):
        pos, vel, frc, step, le = gated.micro.get_state(b)
        shadow.set_state(b, pos, vel, frc, step, le)
    Ld = torch.zeros((nb, 9), dtype=torch.float32, device="cuda")
    st = torch.zeros((nb, 6), dtype=torch.float64, device="cuda")
    Xs, Ts = [], []
    for _ in range(n_steps):
        for sysm in lockstep:
            sysm.step(1, use_graph=True)
        gated.step(1, use_graph=True)
        X = gated.closure_inputs()
        L, _ = gated.exchange()
        Ld.copy_(torch.from_numpy(L))
        shadow.advance(Ld, gated.k_micro, st)
        T = st.cpu().numpy()[:, STRESS_COLS].astype(np.float32)
        if not absolute:
            T = T - X[:, 64:67]
        Xs.append(X)
        Ts.append(T)
    return np.concatenate(Xs), np.concatenate(Ts)


def _rate(cpl, steps):
    import torch
    s = torch.cuda.current_stream()
    cpl.step(2, use_graph=True)  # eager + capture
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    cpl.step(steps, use_graph=True)
    e1.record(s)
    e1.synchronize()
    return steps / (e0.elapsed_time(e1) / 1e3)


def surrogate_vs_plain(warm=20, n_data=150, train_steps=2000, batch=4096, n_eval=60,
                       threshold=0.02, audit_every=50, timing_steps=10, seed=3, alpha=0.01,
                       U_o=0.25, c_factor=10.0, eta_s=0.1, k_micro=50, dt_dpd=0.01, members=5,
                       lr=1e-3, weight_decay=1e-4, cosine=False, nbins=16, thresholds=None,
                       noise_floor=False, absolute=False, warmup_steps=-1, calibrated=False,
                       onpolicy_rounds=0, onpolicy_steps=50, onpolicy_train_steps=None,
                       online_calibration=False, calibration_decay=0.9):
    """Plain LHMM vs surrogate-gated LHMM on the coupled reverse-Poiseuille
    channel.  Two identical systems run the same `warm + n_data` plain steps
    (one collects training pairs); the ensemble trains on the GPU; then both run
    `n_eval` steps (plain vs gated) and the time-averaged y-binned pi_xy and N1
    profiles are compared.  `thresholds` (a list) runs one evaluation window of
    `n_eval` steps per gate threshold, in order, each compared with the same
    window of the plain run.  `noise_floor` adds a third, plain system with
    another DPD seed and reports its profile error against the plain run over
    the same windows: the error two plain runs already differ by.  Returns a
    dict of rates, errors and counts.  `absolute` trains and gates the
    closure on the stress itself from the gradient history (no stress input)
    instead of the increment.  `onpolicy_rounds` > 0 then runs that many
    rounds of `onpolicy_steps` gated steps whose shadow-DPD labels
    (`onpolicy_pairs`) join the training set before the closure trains
    again (onpolicy_train_steps, default train_steps) and, if `calibrated`,
    is recalibrated on the newest on-policy pairs.  `online_calibration`
    lets the gate refit a per-component line from its audited boxes after
    every gated macro step (lhmm_coupled_set_online_calibration, decay
    `calibration_decay`) and applies it to the trusted boxes."""
    kw = dict(alpha=alpha, U_o=U_o, c_factor=c_factor, eta_s=eta_s, k_micro=k_micro,
              dt_dpd=dt_dpd, members=members)
    A, clo_a, cfg, M = _channel(seed=seed, closure_seed=1, **kw)
    B, clo_b, _, _ = _channel(seed=seed, closure_seed=7, **kw)
    systems = [("A", A), ("B", B)]
    C = None
    if noise_floor:
        C, clo_c, _, _ = _channel(seed=seed + 1000, closure_seed=1, **kw)
        systems.append(("C", C))
    A.set_closure(clo_a, threshold=threshold, audit_every=audit_every)
    B.set_closure(clo_b, threshold=threshold, audit_every=audit_every)
    B.set_gate(threshold, audit_every, absolute, warmup_steps)
    t0 = time.perf_counter()
    A.step(warm + n_data, use_graph=True)
    if C is not None:
        C.step(warm + n_data, use_graph=True)
    B.step(warm, use_graph=True)
    X, T = collect_pairs(B, n_data, skip=0, absolute=absolute)
    t_data = time.perf_counter() - t0
    n_fit = X.shape[0] if not calibrated else (X.shape[0] * 9 // 10)  # last 10 %: calibration
    mean, std, scale = normalization(X[:n_fit], T[:n_fit])
    clo_b.set_normalization(mean, std, scale)
    hist, t_train = train(clo_b, X[:n_fit], T[:n_fit], train_steps, batch=batch, lr=lr,
                          weight_decay=weight_decay, log_every=max(1, train_steps // 10),
                          cosine=cosine)
    calib = None
    if calibrated:
        a_c, c_c = calibrate(clo_b, X[n_fit:], T[n_fit:], scale)
        calib = dict(a=a_c.tolist(), c=c_c.tolist())
    if online_calibration:
        B.set_online_calibration(True, calibration_decay)
    B.enable_gate(True)
    n_onpolicy = 0
    if onpolicy_rounds > 0:
        shadow = lhmm.Micro.from_batch(B.micro_params, B.micro_batch)
        lock = [A] + ([C] if C is not None else [])
        for _ in range(onpolicy_rounds):
            B.set_gate(threshold, audit_every, absolute, warmup_steps)
            Xo, To = onpolicy_pairs(B, shadow, onpolicy_steps, absolute, lockstep=lock)
            n_onpolicy += Xo.shape[0]
            n_new = Xo.shape[0] if not calibrated else (Xo.shape[0] * 9 // 10)
            X = np.concatenate([X[:n_fit], Xo[:n_new]])
            T = np.concatenate([T[:n_fit], To[:n_new]])
            n_fit = X.shape[0]
            h2, t2 = train(clo_b, X, T, onpolicy_train_steps or train_steps, batch=batch, lr=lr,
                           weight_decay=weight_decay, seed=1 + n_onpolicy, cosine=cosine)
            t_train += t2
            if calibrated:
                a_c, c_c = calibrate(clo_b, Xo[n_new:], To[n_new:], scale)
                calib = dict(a=a_c.tolist(), c=c_c.tolist())
        shadow.close()
    Ly = cfg["Ly"]
    windows = []
    for thr in (thresholds if thresholds else [threshold]):
        B.set_gate(thr, audit_every, absolute, warmup_steps)
        acc = {name: [np.zeros(nbins), np.zeros(nbins)] for name, _ in systems}
        g_before = B.gate_stats()
        for _ in range(n_eval):
            for name, sysm in systems:
                sysm.step(1, use_graph=True)
                y = sysm.sph.get_state()[0][:, 1]
                _, st = sysm.exchange()
                pxy, n1 = binned_profiles(y, st, Ly, nbins)
                acc[name][0] += pxy / n_eval
                acc[name][1] += n1 / n_eval
        g_after = B.gate_stats()
        w = dict(threshold=thr,
                 stress_error_pxy=rel_l2(acc["B"][0], acc["A"][0]),
                 stress_error_n1=rel_l2(acc["B"][1], acc["A"][1]),
                 dpd_fraction=(g_after["dpd_boxes"] - g_before["dpd_boxes"])
                 / max(1, (g_after["gated_steps"] - g_before["gated_steps"]) * B.n_boxes),
                 profile_pxy_plain=acc["A"][0].tolist(),
                 profile_pxy_surrogate=acc["B"][0].tolist())
        if C is not None:
            w["noise_floor_pxy"] = rel_l2(acc["C"][0], acc["A"][0])
            w["noise_floor_n1"] = rel_l2(acc["C"][1], acc["A"][1])
        windows.append(w)
    gs0 = B.gate_stats()
    rate_plain = _rate(A, timing_steps)
    rate_gated = _rate(B, timing_steps)
    gs = B.gate_stats()
    # the ceiling of the gated step on this system: every box trusted, no
    # audit, so no box runs DPD (SPH substeps, inference and gate only)
    B.set_gate(1e30, 0, absolute, warmup_steps)
    rate_ceiling = _rate(B, timing_steps)
    status = [lhmm.status_string(x.micro.sync(raise_on_error=False)[0]) for x in (A, B)]
    last = windows[-1]
    out = dict(
        device_status_plain=status[0], device_status_surrogate=status[1],
        macro_steps_per_s_plain=rate_plain, macro_steps_per_s_surrogate=rate_gated,
        speedup=rate_gated / rate_plain,
        macro_steps_per_s_no_dpd=rate_ceiling, speedup_ceiling=rate_ceiling / rate_plain,
        stress_error_pxy=last["stress_error_pxy"], stress_error_n1=last["stress_error_n1"],
        dpd_fraction_eval=last["dpd_fraction"],
        dpd_fraction_timed=(gs["dpd_boxes"] - gs0["dpd_boxes"])
        / max(1, (gs["gated_steps"] - gs0["gated_steps"]) * B.n_boxes),
        audit_rel_err=float(np.sqrt(gs["audit_err2"] / max(gs["audit_ref2"], 1e-300))),
        train_pairs=int(X.shape[0]), train_steps=train_steps, batch=batch,
        onpolicy_rounds=onpolicy_rounds, onpolicy_pairs=n_onpolicy,
        train_loss_first=[float(x) for x in hist[0]] if hist else None,
        train_loss_last=[float(x) for x in hist[-1]] if hist else None,
        t_data_s=t_data, t_train_s=t_train, sph_substeps=M, micro_steps=k_micro,
        boxes=B.n_boxes, threshold=last["threshold"], audit_every=audit_every, n_eval=n_eval,
        target="stress" if absolute else "increment", calibration=calib,
        online_calibration=(B.set_online_calibration(-1).tolist() if online_calibration else None),
        windows=windows if len(windows) > 1 else None,
        noise_floor_pxy=last.get("noise_floor_pxy"), noise_floor_n1=last.get("noise_floor_n1"),
        profile_pxy_plain=last["profile_pxy_plain"],
        profile_pxy_surrogate=last["profile_pxy_surrogate"])
    objs = [A, B, clo_a, clo_b] + ([C, clo_c] if C is not None else [])
    for obj in objs:
        obj.close()
    return out


def _cylinder_system(n_fluid, cell, box_beads, U_o, c_factor, eta_s, alpha, k_micro, dt_dpd,
                     seed):
    """The large mixed workload: cylinder-array SPH particles with walls and
    one AFBC box per fluid particle, coupled (autotuned launches)."""
    import torch
    from . import synth
    pos, is_wall, L, dh = synth.cylinder_array(n_fluid_target=n_fluid, radius_frac=0.25, cell=cell)
    n = pos.shape[0]
    n_wall = int(is_wall.sum())
    eta_tot = eta_s + 0.01
    F = 48.0 * eta_tot * U_o / L ** 2
    c = c_factor * U_o
    delta_t = k_micro * dt_dpd
    dt_cfl = 0.25 * min(dh / (1.5 * U_o + c), np.sqrt(dh / F), dh * dh / (2.0 * eta_tot))
    M = int(np.ceil(delta_t / dt_cfl))
    sp = lhmm.sph_params(n, n_wall, Lx=L, Ly=L, h=3 * dh, mass=dh * dh, rho0=1.0, c=c,
                         theta_pb=0.1, eta_s=eta_s, dt=delta_t / M, body_force=(F, 0.0),
                         body_mode=lhmm.SPH_BODY_UNIFORM)
    sph = lhmm.Sph(sp, pos, np.zeros_like(pos))
    edge = (box_beads / synth.DENSITY) ** (1.0 / 3.0)
    batch = synth.make_batch(np.full(n_fluid, edge), np.zeros((n_fluid, 9), np.float32), seed,
                             flow="afbc", n_beads=np.full(n_fluid, box_beads))
    micro = lhmm.Micro.from_batch(lhmm.dpd_params(flow="afbc", seed=seed, alpha=alpha), batch)
    L0 = torch.zeros((n_fluid, 9), dtype=torch.float32, device="cuda")
    micro.autotune(L0, probe_steps=5)
    cpl = lhmm.Coupled(sph, micro, M, k_micro)
    return cpl, sph, micro, batch, L, M, n_wall


def large_mixed_accuracy(n_fluid=16384, cell=16.0, box_beads=1000, U_o=0.25, c_factor=10.0,
                         eta_s=0.1, alpha=0.01, k_micro=50, dt_dpd=0.01, seed=5, warm=20,
                         n_data=60, train_steps=4000, n_eval=100, threshold=0.02,
                         audit_every=50, absolute=False, noise_floor=True, nbins=8,
                         timing_steps=50, weight_decay=0.0, warmup_steps=-1, thresholds=None,
                         calibrated=False, online_calibration=False, calibration_decay=0.9):
    """Surrogate-gated vs plain on the large mixed workload: two identical
    systems (and, with noise_floor, a third plain one with another seed) run
    the same plain steps; one collects pairs and trains its closure; then all
    run n_eval steps and the time-averaged pi_xy and N1 fields, binned on an
    nbins x nbins grid over the cell (fluid particles), are compared.
    `thresholds` (a list) runs one evaluation window per gate threshold, in
    order; `calibrated` holds out the last 10 % of the pairs for the linear
    recalibration of the ensemble output (`calibrate`); `online_calibration`
    lets the gate refit that line from its audits every macro step.  The
    rates are timed at the last threshold.  Returns errors, DPD shares and
    rates."""
    kw = dict(n_fluid=n_fluid, cell=cell, box_beads=box_beads, U_o=U_o, c_factor=c_factor,
              eta_s=eta_s, alpha=alpha, k_micro=k_micro, dt_dpd=dt_dpd)
    A, sphA, microA, batch, Lc, M, n_wall = _cylinder_system(seed=seed, **kw)
    B, sphB, microB, _, _, _, _ = _cylinder_system(seed=seed, **kw)
    systems = [("A", A, sphA), ("B", B, sphB)]
    objs = [A, microA, sphA, B, microB, sphB]
    if noise_floor:
        Cc, sphC, microC, _, _, _, _ = _cylinder_system(seed=seed + 1000, **kw)
        systems.append(("C", Cc, sphC))
        objs += [Cc, microC, sphC]
    clo = lhmm.Closure(members=5, in_dim=N_IN, hidden=256, n_hidden=4, out_dim=N_OUT, seed=seed)
    objs.append(clo)
    B.set_closure(clo, threshold=threshold, audit_every=audit_every)
    B.set_gate(threshold, audit_every, absolute, warmup_steps)
    for name, sysm, _ in systems:
        if name != "B":
            sysm.step(warm + n_data, use_graph=True)
    B.step(warm, use_graph=True)
    X, T = collect_pairs(B, n_data, skip=0, absolute=absolute)
    n_fit = X.shape[0] if not calibrated else (X.shape[0] * 9 // 10)  # last 10 %: calibration
    mean, std, scale = normalization(X[:n_fit], T[:n_fit])
    clo.set_normalization(mean, std, scale)
    _, t_train = train(clo, X[:n_fit], T[:n_fit], train_steps, weight_decay=weight_decay)
    if calibrated:
        calibrate(clo, X[n_fit:], T[n_fit:], scale)
    if online_calibration:
        B.set_online_calibration(True, calibration_decay)
    B.enable_gate(True)
    nf = n_fluid
    windows = []
    for thr in (thresholds if thresholds else [threshold]):
        B.set_gate(thr, audit_every, absolute, warmup_steps)
        g0 = B.gate_stats()
        acc = {name: np.zeros((2, nbins * nbins)) for name, _, _ in systems}
        for _ in range(n_eval):
            for name, sysm, sph in systems:
                sysm.step(1, use_graph=True)
                p = sph.get_state()[0][:nf]
                _, st = sysm.exchange()
                ix = np.minimum((p[:, 0] / Lc * nbins).astype(int), nbins - 1)
                iy = np.minimum((p[:, 1] / Lc * nbins).astype(int), nbins - 1)
                k = ix + nbins * iy
                cnt = np.maximum(np.bincount(k, minlength=nbins * nbins), 1)
                acc[name][0] += np.bincount(k, weights=st[:, 3],
                                            minlength=nbins * nbins) / cnt / n_eval
                acc[name][1] += np.bincount(k, weights=st[:, 0] - st[:, 1],
                                            minlength=nbins * nbins) / cnt / n_eval
        g1 = B.gate_stats()
        w = dict(threshold=thr,
                 stress_error_pxy=rel_l2(acc["B"][0], acc["A"][0]),
                 stress_error_n1=rel_l2(acc["B"][1], acc["A"][1]),
                 dpd_fraction=(g1["dpd_boxes"] - g0["dpd_boxes"])
                 / max(1, (g1["gated_steps"] - g0["gated_steps"]) * nf))
        if noise_floor:
            w["noise_floor_pxy"] = rel_l2(acc["C"][0], acc["A"][0])
            w["noise_floor_n1"] = rel_l2(acc["C"][1], acc["A"][1])
        windows.append(w)
    rate_gated = _rate(B, timing_steps)
    rate_plain = _rate(A, timing_steps)
    last = windows[-1]
    out = dict(workload="periodic cylinder array, %d fluid + %d wall SPH particles, %d-bead AFBC "
                        "boxes, k'=%d, M=%d" % (n_fluid, n_wall, box_beads, k_micro, M),
               target="stress" if absolute else "increment", threshold=last["threshold"],
               train_pairs=int(X.shape[0]), train_steps=train_steps, t_train_s=t_train,
               n_eval=n_eval, nbins=nbins,
               stress_error_pxy=last["stress_error_pxy"], stress_error_n1=last["stress_error_n1"],
               dpd_fraction=last["dpd_fraction"],
               macro_steps_per_s_plain=rate_plain, macro_steps_per_s_surrogate=rate_gated,
               speedup=rate_gated / rate_plain,
               online_calibration=(B.set_online_calibration(-1).tolist()
                                   if online_calibration else None),
               windows=windows if len(windows) > 1 else None,
               device_status=lhmm.status_string(microB.sync(raise_on_error=False)[0]))
    if noise_floor:
        out["noise_floor_pxy"] = last["noise_floor_pxy"]
        out["noise_floor_n1"] = last["noise_floor_n1"]
    for o in objs:
        o.close()
    return out


def large_mixed_run(n_fluid=16384, cell=16.0, box_beads=1000, U_o=0.25, c_factor=10.0,
                    eta_s=0.1, alpha=0.01, k_micro=50, dt_dpd=0.01, seed=5, warm=10, n_data=30,
                    train_steps=2000, timing_steps=10, threshold=0.02, audit_every=50):
    """Periodic array of cylinders (radius 0.25 of the cell width) with wall
    particles, one box of box_beads beads per fluid particle; plain macro
    steps, then pairs, closure training and surrogate-gated macro steps on the
    same system (CUDA graphs, the autotuned launch plan, persistent gated
    launches).  Returns rates and counts."""
    import torch
    from . import synth
    t_setup = time.perf_counter()
    pos, is_wall, L, dh = synth.cylinder_array(n_fluid_target=n_fluid, radius_frac=0.25, cell=cell)
    n = pos.shape[0]
    n_wall = int(is_wall.sum())
    eta_tot = eta_s + 0.01
    F = 48.0 * eta_tot * U_o / L ** 2
    c = c_factor * U_o
    delta_t = k_micro * dt_dpd
    dt_cfl = 0.25 * min(dh / (1.5 * U_o + c), np.sqrt(dh / F), dh * dh / (2.0 * eta_tot))
    M = int(np.ceil(delta_t / dt_cfl))
    sp = lhmm.sph_params(n, n_wall, Lx=L, Ly=L, h=3 * dh, mass=dh * dh, rho0=1.0, c=c,
                         theta_pb=0.1, eta_s=eta_s, dt=delta_t / M, body_force=(F, 0.0),
                         body_mode=lhmm.SPH_BODY_UNIFORM)
    sph = lhmm.Sph(sp, pos, np.zeros_like(pos))
    edge = (box_beads / synth.DENSITY) ** (1.0 / 3.0)
    batch = synth.make_batch(np.full(n_fluid, edge), np.zeros((n_fluid, 9), np.float32), seed,
                             flow="afbc", n_beads=np.full(n_fluid, box_beads))
    micro = lhmm.Micro.from_batch(lhmm.dpd_params(flow="afbc", seed=seed, alpha=alpha), batch)
    L0 = torch.zeros((n_fluid, 9), dtype=torch.float32, device="cuda")
    micro.autotune(L0, probe_steps=5)
    cpl = lhmm.Coupled(sph, micro, M, k_micro)
    clo = lhmm.Closure(members=5, in_dim=N_IN, hidden=256, n_hidden=4, out_dim=N_OUT, seed=seed)
    cpl.set_closure(clo, threshold=threshold, audit_every=audit_every)
    t_setup = time.perf_counter() - t_setup
    cpl.step(warm, use_graph=True)
    rate_plain = _rate(cpl, timing_steps)
    X, T = collect_pairs(cpl, n_data, skip=HIST)
    mean, std, scale = normalization(X, T)
    clo.set_normalization(mean, std, scale)
    _, t_train = train(clo, X, T, train_steps)
    cpl.enable_gate(True)
    g0 = cpl.gate_stats()
    rate_gated = _rate(cpl, timing_steps)
    g1 = cpl.gate_stats()
    cpl.set_gate(1e30, 0)  # ceiling: every box trusted, none on DPD
    rate_ceiling = _rate(cpl, min(timing_steps, 50))
    status = lhmm.status_string(micro.sync(raise_on_error=False)[0])
    out = dict(workload="periodic cylinder array: cell %.0f, radius 0.25 cell, %d fluid + %d wall SPH "
                        "particles, %d-bead AFBC boxes (%d beads), k'=%d, M=%d"
                        % (L, n_fluid, n_wall, box_beads, batch.total_beads, k_micro, M),
               macro_steps_per_s_plain=rate_plain, macro_steps_per_s_surrogate=rate_gated,
               speedup=rate_gated / rate_plain,
               macro_steps_per_s_no_dpd=rate_ceiling, speedup_ceiling=rate_ceiling / rate_plain,
               bead_steps_per_s_plain=rate_plain * batch.total_beads * k_micro,
               dpd_fraction=(g1["dpd_boxes"] - g0["dpd_boxes"])
               / max(1, (g1["gated_steps"] - g0["gated_steps"]) * n_fluid),
               train_pairs=int(X.shape[0]), train_steps=train_steps, t_train_s=t_train,
               t_setup_s=t_setup, device_status=status, launch_plan=micro.plan())
    for o in (cpl, clo, micro, sph):
        o.close()
    return out
