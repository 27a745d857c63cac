"""The coupled LHMM on reverse-Poiseuille flow (Sec. 6.1) satisfies the exact
momentum balance: in the steady state the solvent + polymer shear stress is
F rho (y - L_y/4) in the lower half (Eq. RPF, read as sigma_xy = -tau_xy),
whatever the polymer closure.  A small, fast version of the paper's set-up:
20 x 20 SPH particles (Lucy, h = 4 dh), 2D melt boxes of 12 x 12 (Table 1
parameters, N_d = 8), a larger solvent viscosity so that the flow converges
in ~50 macro steps, and a polymer share of ~30 %."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def test_coupled_rpf_matches_exact_shear_stress():
    from paper_2512_13267_gb300 import flows
    out = flows.rpf_paper(F=2e-2, chain_len=8, alpha=1e-2, n_macro=600, n_avg=450, box_edge=12.0,
                          nbins=10, eta_s=0.2, dh=0.2, dt_sph=0.01, c=1.0, timing_steps=5)
    assert out["device_status"] == "ok"
    sig, ex = np.array(out["sigma_total"]), np.array(out["sigma_exact"])
    # 20 particles across L_y with h = 4 dh = L_y / 5 smooth the profile's
    # kinks at y = 0 and L_y / 2: a resolution error of 5-8 % of tau_max that
    # stays when the average is made four times longer (the paper-size runs
    # reach 1-3 %)
    assert out["max_abs_error_over_tau_max"] < 0.10, (sig, ex)
    assert out["rel_l2_error"] < 0.09, out["rel_l2_error"]
    # the polymer carries a real share of the stress, with the flow's sign
    pol = np.array(out["sigma_polymer"])
    assert out["polymer_share"] > 0.1
    assert np.all(np.sign(pol[[0, 1, 3, 4]]) == np.sign(ex[[0, 1, 3, 4]]))


def test_porous_medium_coupled_step_runs_with_walls():
    # the paper-scale porous-medium workload at small boxes: 17 obstacles with
    # wall particles, one 2D melt box per fluid particle, graph-replayed steps
    from paper_2512_13267_gb300 import flows
    out = flows.rpm_paper_rate(steps=1, warmup=1, chain_len=8, box_edge=12.0,
                               distinct_states=8)
    assert out["device_status"] == "ok"
    assert out["value"] > 0.0
    assert out["wall_particles"] > 0 and out["boxes"] == out["fluid_particles"]
