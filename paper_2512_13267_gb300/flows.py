"""Coupled LHMM runs of the paper's reverse-Poiseuille benchmark (Sec. 6.1).

Reverse-Poiseuille flow (RPF): a periodic square of side L_y, body force +F
(per unit mass) in the upper half and -F in the lower half.  Momentum
balance fixes the steady total shear stress exactly, whatever the polymer
closure:
    tau_xy(y) = F rho (L_y/4 - y)       for y <  L_y/2,
    tau_xy(y) = F rho (y - 3 L_y/4)     for y >= L_y/2     (Eq. RPF),
where tau is the momentum flux, minus the Cauchy shear stress sigma_xy that
the momentum equation dv/dt = div(sigma)/rho + f uses (reading R14: steady
d sigma_xy/dy = -rho f_x with zero mean gives sigma_xy = F rho (y - L_y/4) in
the lower half).  The time-averaged solvent + polymer sigma_xy of a
converged coupled run is checked against -tau_xy.  The set-up follows
the paper: L_x = L_y = 4, dh = 0.1 (40 x 40 particles), Lucy kernel with
h = 4 dh, rho = 1, eta_s = 0.02, Delta t_SPH = 0.04, coupling interval
delta t = 0.32 = 64 DPD steps of 0.005, one 2D melt box per particle
(Table 1 parameters, AFBC squares).  The paper's boxes are 76 x 76; here
they are box_edge x box_edge (the engine keeps a box in one SM's shared
memory).
"""
import time

import numpy as np

from . import lhmm, rheometry, synth


def rpf_exact_shear_stress(y, F, Ly, rho=1.0):
    """Eq. RPF: the steady total shear stress of reverse-Poiseuille flow."""
    y = np.asarray(y, dtype=np.float64)
    return np.where(y < 0.5 * Ly, F * rho * (0.25 * Ly - y), F * rho * (y - 0.75 * Ly))


def _rpf_system(F, chain_len, alpha, box_edge, seed, c, eta_s, exclude_bonds, dh, dt_sph):
    """SPH particles, micro boxes and the coupled handle of the RPF set-up."""
    import torch
    Ly = Lx = 4.0
    n_side = int(round(Ly / dh))
    pos = synth.sph_lattice(n_side, n_side, Lx, Ly)
    n = pos.shape[0]
    k_micro = 64
    M = int(round(k_micro * rheometry.PAPER_2D["dt"] / dt_sph))  # 0.32 / 0.04 = 8
    sp = lhmm.sph_params(n, 0, Lx=Lx, Ly=Ly, h=4.0 * dh, mass=dh * dh, rho0=1.0, c=c,
                         theta_pb=0.1, eta_s=eta_s, dt=dt_sph, kernel=lhmm.SPH_LUCY,
                         body_force=(F, 0.0), body_mode=lhmm.SPH_BODY_REVERSE_POISEUILLE)
    sph = lhmm.Sph(sp, pos, np.zeros_like(pos))
    nb = int(round(4 * box_edge * box_edge))
    nb -= nb % chain_len
    batch = synth.make_batch(np.full(n, box_edge), np.zeros((n, 9), np.float32), seed,
                             flow="afbc", chain_len=chain_len, fraction=1.0,
                             n_beads=np.full(n, nb), dim=2)
    micro = lhmm.Micro.from_batch(
        lhmm.dpd_params(flow="afbc", seed=seed, dim=2, alpha=alpha, exclude_bonds=exclude_bonds,
                        **rheometry.PAPER_2D), batch)
    L0 = torch.zeros((n, 9), dtype=torch.float32, device="cuda")
    micro.autotune(L0, probe_steps=8)
    cpl = lhmm.Coupled(sph, micro, M, k_micro)
    return sph, micro, cpl, batch, M, k_micro, Ly


def _rate(cpl, steps):
    import torch
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    cpl.step(steps, use_graph=True)
    e1.record(s)
    e1.synchronize()
    return steps / (e0.elapsed_time(e1) / 1e3)


def rpf_paper_rate(steps=20, warmup=3, F=1e-3, chain_len=8, alpha=1e-4, box_edge=20.0, seed=3):
    """Macro-steps/s of the paper's RPF set-up (graph-replayed macro steps
    after `warmup` untimed ones), without the convergence run."""
    sph, micro, cpl, batch, M, k_micro, _ = _rpf_system(F, chain_len, alpha, box_edge, seed, 0.25,
                                                        0.02, 0, 0.1, 0.04)
    cpl.step(warmup, use_graph=True)
    rate = _rate(cpl, steps)
    status = lhmm.status_string(micro.sync(raise_on_error=False)[0])
    out = dict(metric="LHMM macro-steps/s (plain DPD closure), paper's RPF set-up",
               value=rate, unit="macro-steps/s", steps=steps, warmup=warmup,
               sph_particles=int(batch.n_boxes), sph_substeps=M, micro_steps=k_micro,
               boxes=batch.n_boxes, beads=int(batch.total_beads),
               bead_steps_per_s=rate * batch.total_beads * k_micro, device_status=status,
               workload="reverse-Poiseuille 40x40 SPH (Lucy h=4dh, eta_s=0.02, dt_SPH=0.04) x "
                        "2D N_d=%d melt boxes of %d beads (Table 1, AFBC), 64 DPD steps per "
                        "macro step, F=%g" % (chain_len, int(batch.n_beads[0]), F))
    for o in (cpl, micro, sph):
        o.close()
    return out


def rpf_paper(F=1e-3, chain_len=8, alpha=1e-4, n_macro=1000, n_avg=300, box_edge=20.0,
              nbins=20, seed=3, c=0.25, eta_s=0.02, exclude_bonds=0, timing_steps=50,
              dh=0.1, dt_sph=0.04):
    """Run the coupled RPF of Sec. 6.1 and compare the time-averaged binned
    total shear stress sigma_xy = eta_s (L_xy + L_yx) + pi_xy (pi as the SPH
    momentum equation uses it) with -tau_xy of Eq. RPF over the last n_avg of
    n_macro macro steps.  Returns the profiles, the relative L2 error, the
    largest error over tau_max = F rho L_y / 4, and macro-steps/s."""
    sph, micro, cpl, batch, M, k_micro, Ly = _rpf_system(F, chain_len, alpha, box_edge, seed, c,
                                                         eta_s, exclude_bonds, dh, dt_sph)
    n = batch.n_boxes
    nb = int(batch.n_beads[0])
    t0 = time.perf_counter()
    cpl.step(n_macro - n_avg, use_graph=True)
    edges = np.linspace(0.0, Ly, nbins + 1)
    acc = np.zeros(nbins)
    acc_p = np.zeros(nbins)
    cnt = np.zeros(nbins)
    for _ in range(n_avg):
        cpl.step(1, use_graph=True)
        y = sph.get_state()[0][:, 1]
        Lg, st = cpl.exchange()
        tau = eta_s * (Lg[:, 1] + Lg[:, 3]) + st[:, 3]
        k = np.clip(np.searchsorted(edges, y, side="right") - 1, 0, nbins - 1)
        acc += np.bincount(k, weights=tau, minlength=nbins)
        acc_p += np.bincount(k, weights=st[:, 3], minlength=nbins)
        cnt += np.bincount(k, minlength=nbins)
    wall = time.perf_counter() - t0
    prof = acc / np.maximum(cnt, 1)
    prof_p = acc_p / np.maximum(cnt, 1)
    yc = 0.5 * (edges[1:] + edges[:-1])
    exact = -rpf_exact_shear_stress(yc, F, Ly)  # sigma_xy = -tau_xy
    tau_max = F * Ly / 4.0
    rate = _rate(cpl, timing_steps)
    status = lhmm.status_string(micro.sync(raise_on_error=False)[0])
    out = dict(F=F, chain_len=chain_len, alpha=alpha, particles=n, box_beads=nb,
               beads=int(batch.total_beads), sph_substeps=M, micro_steps=k_micro,
               n_macro=n_macro, n_avg=n_avg, y=yc.tolist(), sigma_total=prof.tolist(),
               sigma_exact=exact.tolist(), sigma_polymer=prof_p.tolist(),
               rel_l2_error=float(np.linalg.norm(prof - exact) / np.linalg.norm(exact)),
               max_abs_error_over_tau_max=float(np.abs(prof - exact).max() / tau_max),
               polymer_share=float(np.abs(prof_p).sum() / max(np.abs(prof).sum(), 1e-30)),
               macro_steps_per_s=rate,
               bead_steps_per_s=rate * batch.total_beads * k_micro, wall_s=wall,
               device_status=status)
    for o in (cpl, micro, sph):
        o.close()
    return out


def rpm_paper_rate(steps=3, warmup=1, chain_len=16, box_edge=76.0, F=1e-3, alpha=1e-4,
                   eta_s=0.02, c=0.5, distinct_states=64, seed=5):
    """Macro-steps/s at the scale of the paper's random-porous-medium run
    (Sec. 6.3): a periodic 12 x 4 box with 17 cylinders at porosity 0.792
    (synthetic placement: the paper's obstacle table is not available),
    dh = 1/16, Lucy kernel h = 4 dh, delta_t = 0.125 = 25 DPD steps of 0.005,
    M = 50 SPH substeps of 2.5e-3, and one 2D melt box of box_edge^2 * 4 beads
    of N_d = chain_len chains (Table 1 parameters, AFBC) per fluid particle.
    Boxes start from `distinct_states` different initial states repeated
    (their random streams differ by box id); this only shortens set-up.
    Times graph-replayed macro steps after `warmup` untimed ones."""
    import torch
    pos, is_wall, Lx, Ly, dh, _, _ = synth.random_porous_medium(dh=1.0 / 16.0, seed=seed)
    n = pos.shape[0]
    n_wall = int(is_wall.sum())
    n_fluid = n - n_wall
    k_micro = 25
    M = 50
    sp = lhmm.sph_params(n, n_wall, Lx=Lx, Ly=Ly, h=4.0 * dh, mass=dh * dh, rho0=1.0, c=c,
                         theta_pb=0.1, eta_s=eta_s, dt=k_micro * rheometry.PAPER_2D["dt"] / M,
                         kernel=lhmm.SPH_LUCY, body_force=(F, 0.0),
                         body_mode=lhmm.SPH_BODY_UNIFORM)
    sph = lhmm.Sph(sp, pos, np.zeros_like(pos))
    nb = int(round(4 * box_edge * box_edge))
    nb -= nb % chain_len
    batch = synth.make_batch(np.full(n_fluid, box_edge), np.zeros((n_fluid, 9), np.float32),
                             seed, flow="afbc", chain_len=chain_len, fraction=1.0,
                             n_beads=np.full(n_fluid, nb), dim=2, with_state=False)
    reps = -(-n_fluid // distinct_states)
    ps, vs = [], []
    for b in range(min(distinct_states, n_fluid)):
        p, v = synth.initial_box_state(batch.edges[b].astype(np.float64), nb, seed, b,
                                       L=batch.L[b], flow="afbc", dim=2)
        ps.append(p)
        vs.append(v)
    batch.pos = np.tile(np.concatenate(ps), (reps, 1))[:batch.total_beads]
    batch.vel = np.tile(np.concatenate(vs), (reps, 1))[:batch.total_beads]
    t0 = time.perf_counter()
    micro = lhmm.Micro.from_batch(
        lhmm.dpd_params(flow="afbc", seed=seed, dim=2, alpha=alpha, **rheometry.PAPER_2D), batch)
    batch.pos = batch.vel = None
    L0 = torch.zeros((n_fluid, 9), dtype=torch.float32, device="cuda")
    micro.autotune(L0, probe_steps=5)
    cpl = lhmm.Coupled(sph, micro, M, k_micro)
    t_setup = time.perf_counter() - t0
    cpl.step(warmup, use_graph=True)
    rate = _rate(cpl, steps)
    status = lhmm.status_string(micro.sync(raise_on_error=False)[0])
    beads = int(batch.total_beads)
    out = dict(metric="LHMM macro-steps/s (plain DPD closure), paper-scale porous medium",
               value=rate, unit="macro-steps/s", steps=steps, warmup=warmup,
               sph_particles=n, fluid_particles=n_fluid, wall_particles=n_wall,
               sph_substeps=M, micro_steps=k_micro, boxes=n_fluid, beads=beads,
               bead_steps_per_s=rate * beads * k_micro, s_per_macro_step=1.0 / rate,
               setup_s=t_setup, plan=micro.plan(), device_status=status,
               workload="random porous medium 12x4, 17 cylinders, porosity 0.792, dh=1/16 "
                        "(Lucy h=4dh) x 2D N_d=%d melt boxes of %d beads (AFBC), "
                        "k'=25, M=50" % (chain_len, nb))
    for o in (cpl, micro, sph):
        o.close()
    return out
