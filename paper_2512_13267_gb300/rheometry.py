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
