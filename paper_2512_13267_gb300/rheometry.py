"""Virtual rheometry of the paper's 2D polymer melts on the batched engine.

The paper characterises its micro model (Table 1 parameters, number density
4 per area, melts of N_d-bead FENE chains) by imposing steady shear on a
micro-domain and reading the IK stress: the polymeric shear viscosity
eta(gdot) = pi_xy / gdot, fitted by Carreau-Yasuda (Sec. 5.1, Table 3), and
the first normal stress coefficient psi_1 = N_1 / gdot^2 with
N_1 = pi_xx - pi_yy (Sec. 5.1.1).  Here every (shear rate, replica) pair is
one periodic Lees-Edwards box of the batch (reading R12: homogeneous shear by
sliding images instead of the AFBC rheometer; both impose the same bulk
flow), all advanced together.
"""
import time

import numpy as np

from . import lhmm, synth

# Table 1 of the paper
PAPER_2D = dict(a_ij=25.0, gamma=4.5, sigma=3.0, kBT=1.0, rc=1.0, H_fene=50.0, R0=1.5,
                dt=0.005, mass=1.0)


def carreau_yasuda(gdot, eta0, eta_inf, lam, a, n):
    """eta(gdot) = eta_inf + (eta0 - eta_inf) (1 + (lam gdot)^a)^((n - 1)/a)."""
    g = np.asarray(gdot, dtype=np.float64)
    return eta_inf + (eta0 - eta_inf) * (1.0 + (lam * g) ** a) ** ((n - 1.0) / a)


def fit_carreau_yasuda(gdot, eta, eta_se=None, fix_eta_inf=None, fix_a=None, fix_n=None):
    """Least-squares Carreau-Yasuda fit (Sec. 5.1, appendix on the CY model)
    of eta(gdot), in log eta with weights from the standard errors when given.
    Returns dict(eta0, eta_inf, lam, a, n, rms_log_residual).  fix_eta_inf
    pins eta_inf (the plateau at high rates is often outside the data);
    fix_a / fix_n pin the transition sharpness and the power-law index, so
    that with the paper's shape parameters only eta0 and the onset time lam
    are fitted (over two decades of rate lam otherwise trades off against
    n and eta_inf)."""
    from scipy.optimize import least_squares
    g = np.asarray(gdot, dtype=np.float64)
    y = np.asarray(eta, dtype=np.float64)
    w = np.ones_like(y) if eta_se is None else y / np.maximum(np.asarray(eta_se, np.float64),
                                                              1e-3 * y)
    w = w / w.mean()
    # free parameters in order: log eta0, log(lam median(g)), a, n, log(eta_inf / eta0)
    names = ["eta0", "lam", "a", "n", "inf"]
    fixed = {"a": fix_a, "n": fix_n, "inf": fix_eta_inf}
    free = [k for k in names if fixed.get(k) is None]
    q0 = {"eta0": np.log(y.max() * 1.2), "lam": 0.0, "a": 1.0, "n": 0.4, "inf": np.log(0.05)}
    lo = {"eta0": np.log(y.max() * 0.5), "lam": np.log(1e-2 / g.max() * np.median(g)), "a": 0.2,
          "n": 0.0, "inf": np.log(1e-4)}
    hi = {"eta0": np.log(y.max() * 20.0), "lam": np.log(1e3 / g.min() * np.median(g)), "a": 3.0,
          "n": 0.99, "inf": np.log(0.5)}

    def unpack(q):
        v = dict(zip(free, q))
        eta0 = np.exp(v["eta0"])
        lam = np.exp(v["lam"]) / np.median(g)
        a = v["a"] if fix_a is None else fix_a
        n = v["n"] if fix_n is None else fix_n
        eta_inf = fix_eta_inf if fix_eta_inf is not None else np.exp(v["inf"]) * eta0
        return eta0, eta_inf, lam, a, n

    def resid(q):
        eta0, eta_inf, lam, a, n = unpack(q)
        return w * (np.log(carreau_yasuda(g, eta0, eta_inf, lam, a, n)) - np.log(y))

    lo_v = np.array([lo[k] for k in free])
    hi_v = np.array([hi[k] for k in free])
    best = None
    for lam0 in (0.3, 1.0, 3.0):  # a few starts in lambda
        q = np.array([q0[k] if k != "lam" else np.log(lam0) for k in free])
        q = np.clip(q, lo_v + 1e-9, hi_v - 1e-9)
        r = least_squares(resid, q, bounds=(lo_v, hi_v))
        if best is None or r.cost < best.cost:
            best = r
    eta0, eta_inf, lam, a, n = unpack(best.x)
    rms = float(np.sqrt(np.mean((best.fun / w) ** 2)))
    return dict(eta0=float(eta0), eta_inf=float(eta_inf), lam=float(lam), a=float(a), n=float(n),
                rms_log_residual=rms)


def melt_viscosity(chain_len, shear_rates, replicas=32, edge=20.0, equil_time=None,
                   sample_time=None, call_steps=1000, seed=11, dpd_on_bonded=1,
                   exclude_bonds=0):
    """Steady-shear viscosity and psi_1 of a 2D melt of chain_len-bead chains.

    Returns per shear rate the replica mean and standard error of eta and
    psi_1, plus run counts.  equil_time / sample_time (DPD time units)
    default to 5 and 10 Rouse-scaled relaxation times of the chain
    (23.5 (chain_len / 4)^2, the N_d = 4 value of Table 3 with Rouse scaling),
    at least 100 and 200.  dpd_on_bonded = 0 drops the DPD pair forces
    between bonded neighbours, exclude_bonds = K those of beads of one chain
    up to K bonds apart (reading R5's alternatives)."""
    import torch
    rates = np.asarray(shear_rates, dtype=np.float64)
    lam_guess = 23.5 * (chain_len / 4.0) ** 2
    equil_time = max(100.0, 5 * lam_guess) if equil_time is None else equil_time
    sample_time = max(200.0, 10 * lam_guess) if sample_time is None else sample_time
    dt = PAPER_2D["dt"]
    n_equil = int(np.ceil(equil_time / dt / call_steps))
    n_sample = int(np.ceil(sample_time / dt / call_steps))
    batch = synth.melt_rheometer_batch(chain_len, rates, replicas, edge=edge, seed=seed)
    params = lhmm.dpd_params(flow="lees_edwards", seed=seed, dim=2, dpd_on_bonded=dpd_on_bonded,
                             exclude_bonds=exclude_bonds, **PAPER_2D)
    t0 = time.perf_counter()
    m = lhmm.Micro.from_batch(params, batch)
    L = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    acc = torch.zeros_like(st)
    for _ in range(n_equil):
        m.advance(L, call_steps, st)
    for _ in range(n_sample):
        m.advance(L, call_steps, st)
        acc += st
    status = m.sync(raise_on_error=False)[0]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    mean = (acc / n_sample).cpu().numpy().reshape(len(rates), replicas, 6)
    g = rates[:, None]
    eta = mean[:, :, 3] / g
    psi1 = (mean[:, :, 0] - mean[:, :, 1]) / g ** 2
    se = lambda x: x.std(axis=1, ddof=1) / np.sqrt(x.shape[1])
    m.close()
    return dict(chain_len=chain_len, shear_rates=rates.tolist(), replicas=replicas, edge=edge,
                dpd_on_bonded=dpd_on_bonded, exclude_bonds=exclude_bonds,
                beads_per_box=int(batch.n_beads[0]), boxes=batch.n_boxes,
                eta=eta.mean(axis=1).tolist(), eta_se=se(eta).tolist(),
                psi1=psi1.mean(axis=1).tolist(), psi1_se=se(psi1).tolist(),
                equil_steps=n_equil * call_steps, sample_steps=n_sample * call_steps,
                bead_steps=int(batch.total_beads) * (n_equil + n_sample) * call_steps,
                wall_s=wall, device_status=lhmm.status_string(status))


def stress_relaxation(chain_len, shear_rate, replicas=64, edge=20.0, shear_time=None,
                      relax_time=None, sample_time=1.0, seed=13, exclude_bonds=0,
                      rheometer="lees_edwards", afbc_mode=0):
    """Recovery test (Sec. 5.2): steady shear at shear_rate for shear_time,
    then the shear is removed and the replica-averaged pi_xy is recorded in
    windows of sample_time; G(t) = <pi_xy(t)> / gamma with gamma the total
    applied strain shear_rate * shear_time (the paper's definition).
    rheometer = "lees_edwards": periodic boxes sheared by sliding images;
    "afbc": the paper's rheometer, square boxes sheared through the AFBC
    shell (L_xy = shear_rate, then L = 0, which holds the shell at rest) with
    the stress of the core."""
    import torch
    dt = PAPER_2D["dt"]
    lam_guess = 23.5 * (chain_len / 4.0) ** 2
    shear_time = max(100.0, 5 * lam_guess) if shear_time is None else shear_time
    relax_time = max(100.0, 5 * lam_guess) if relax_time is None else relax_time
    if rheometer == "afbc":
        Lh = np.zeros((replicas, 9), np.float32)
        Lh[:, 1] = shear_rate
        n = int(round(synth.DENSITY_PAPER_2D * edge * edge))
        n -= n % chain_len
        batch = synth.make_batch(np.full(replicas, edge), Lh, seed, flow="afbc",
                                 chain_len=chain_len, fraction=1.0, n_beads=np.full(replicas, n),
                                 dim=2)
        params = lhmm.dpd_params(flow="afbc", seed=seed, dim=2, exclude_bonds=exclude_bonds,
                                 afbc_mode=afbc_mode, **PAPER_2D)
    elif rheometer == "lees_edwards":
        batch = synth.melt_rheometer_batch(chain_len, [shear_rate], replicas, edge=edge, seed=seed)
        params = lhmm.dpd_params(flow="lees_edwards", seed=seed, dim=2,
                                 exclude_bonds=exclude_bonds, **PAPER_2D)
    else:
        raise ValueError("rheometer must be 'lees_edwards' or 'afbc'")
    m = lhmm.Micro.from_batch(params, batch)
    L = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    chunk = 1000
    n_shear = int(np.ceil(shear_time / dt / chunk))
    for _ in range(n_shear):
        m.advance(L, chunk, st)
    sheared = st.mean(dim=0).cpu().numpy()
    L0 = torch.zeros_like(L)
    k = max(1, int(round(sample_time / dt)))
    n_rel = int(np.ceil(relax_time / (k * dt)))
    t, pxy, se = [], [], []
    for s in range(n_rel):
        m.advance(L0, k, st)
        x = st[:, 3].cpu().numpy()
        t.append((s + 0.5) * k * dt)
        pxy.append(float(x.mean()))
        se.append(float(x.std(ddof=1) / np.sqrt(len(x))))
    status = lhmm.status_string(m.sync(raise_on_error=False)[0])
    m.close()
    gamma = shear_rate * n_shear * chunk * dt
    return dict(chain_len=chain_len, shear_rate=shear_rate, replicas=replicas, edge=edge,
                rheometer=rheometer, strain=gamma, steady_pi_xy=float(sheared[3]), t=t,
                pi_xy=pxy, pi_xy_se=se,
                G=[p / gamma for p in pxy], device_status=status)


def planar_extension(chain_len, rates, replicas=32, edge=36.0, equil_time=None,
                     sample_time=None, call_steps=1000, seed=17, exclude_bonds=0,
                     mode="extension", afbc_mode=0):
    """Steady planar extension L = diag(e, -e) imposed through the AFBC shell
    of 2D melt boxes; planar extensional viscosity eta_P = (pi_xx - pi_yy)/e
    from the core's IK stress.  For a Newtonian liquid eta_P = 4 eta (the
    planar Trouton ratio), the low-rate check against the shear viscosity.
    mode = "shear" imposes simple shear L_xy = rate through the same AFBC
    shell instead and returns eta = pi_xy / rate as eta_P (to set against the
    Lees-Edwards rheometer)."""
    import torch
    rates = np.asarray(rates, dtype=np.float64)
    dt = PAPER_2D["dt"]
    lam_guess = 23.5 * (chain_len / 4.0) ** 2
    equil_time = max(100.0, 5 * lam_guess) if equil_time is None else equil_time
    sample_time = max(200.0, 10 * lam_guess) if sample_time is None else sample_time
    e = np.repeat(rates, int(replicas))
    B = e.shape[0]
    L = np.zeros((B, 9), np.float32)
    if mode == "shear":
        L[:, 1] = e
    else:
        L[:, 0] = e
        L[:, 4] = -e
    n = int(round(synth.DENSITY_PAPER_2D * edge * edge))
    n -= n % chain_len
    batch = synth.make_batch(np.full(B, edge), L, seed, flow="afbc", chain_len=chain_len,
                             fraction=1.0, n_beads=np.full(B, n), dim=2)
    params = lhmm.dpd_params(flow="afbc", seed=seed, dim=2, exclude_bonds=exclude_bonds,
                             afbc_mode=afbc_mode, **PAPER_2D)
    t0 = time.perf_counter()
    m = lhmm.Micro.from_batch(params, batch)
    Ld = torch.from_numpy(L).cuda()
    st = torch.zeros((B, 6), dtype=torch.float64, device="cuda")
    acc = torch.zeros_like(st)
    n_equil = int(np.ceil(equil_time / dt / call_steps))
    n_sample = int(np.ceil(sample_time / dt / call_steps))
    for _ in range(n_equil):
        m.advance(Ld, call_steps, st)
    for _ in range(n_sample):
        m.advance(Ld, call_steps, st)
        acc += st
    status = lhmm.status_string(m.sync(raise_on_error=False)[0])
    mean = (acc / n_sample).cpu().numpy().reshape(len(rates), replicas, 6)
    if mode == "shear":
        etaP = mean[:, :, 3] / rates[:, None]
    else:
        etaP = (mean[:, :, 0] - mean[:, :, 1]) / rates[:, None]
    m.close()
    se = lambda x: (x.std(axis=1, ddof=1) / np.sqrt(replicas)).tolist()
    out = dict(chain_len=chain_len, rates=rates.tolist(), replicas=replicas, edge=edge,
               mode=mode, afbc_mode=afbc_mode, beads_per_box=n,
               eta_P=etaP.mean(axis=1).tolist(), eta_P_se=se(etaP),
               wall_s=time.perf_counter() - t0, device_status=status)
    if mode == "shear":  # first normal stress coefficient psi_1 = N_1 / gdot^2
        psi1 = (mean[:, :, 0] - mean[:, :, 1]) / rates[:, None] ** 2
        out.update(psi1=psi1.mean(axis=1).tolist(), psi1_se=se(psi1))
    return out


def relaxation_time(t, g, g_se, t_min=0.0, snr=3.0):
    """Relaxation time of a stress decay g(t) after the flow stops (g = G(t)
    or pi_xy(t); only its shape matters), from the samples with t >= t_min
    that stand snr standard errors above zero:
      lam_tail  = -1 / slope of a weighted straight-line fit of log g on t
                  (the terminal, longest relaxation time);
      lam_moment = int t g dt / int g dt over the same samples (the mean
                  relaxation time of the decay; a single exponential gives
                  its time constant, exactly as the window grows).
    Returns dict(lam_tail, lam_tail_se, lam_moment, n_points, t_max)."""
    t = np.asarray(t, np.float64)
    g = np.asarray(g, np.float64)
    se = np.maximum(np.asarray(g_se, np.float64), 1e-300)
    keep = (t >= t_min) & (g > snr * se)
    # the usable decay ends at the first sample that drops into the noise
    idx = np.flatnonzero(t >= t_min)
    end = idx[0] if idx.size else len(t)
    while end < len(t) and g[end] > snr * se[end]:
        end += 1
    keep &= np.arange(len(t)) < end
    tt, gg, ss = t[keep], g[keep], se[keep]
    if tt.size < 3:
        return dict(lam_tail=float("nan"), lam_tail_se=float("nan"),
                    lam_moment=float("nan"), n_points=int(tt.size), t_max=float("nan"))
    w = (gg / ss) ** 2  # var(log g) ~ (se / g)^2
    A = np.stack([np.ones_like(tt), tt], axis=1)
    cov = np.linalg.inv(A.T @ (A * w[:, None]))
    coef = cov @ (A.T @ (w * np.log(gg)))
    slope, slope_se = coef[1], np.sqrt(cov[1, 1])
    lam = -1.0 / slope if slope < 0 else float("inf")
    lam_se = slope_se / slope ** 2 if slope < 0 else float("inf")
    num = np.trapezoid(tt * gg, tt)
    den = np.trapezoid(gg, tt)
    return dict(lam_tail=float(lam), lam_tail_se=float(lam_se),
                lam_moment=float(num / den - tt[0]), n_points=int(tt.size), t_max=float(tt[-1]))
