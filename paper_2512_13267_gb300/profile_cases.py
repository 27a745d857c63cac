"""Fixed, small invocations of each kernel family for profiling.

    python -m paper_2512_13267_gb300.profile_cases micro   # 304 boxes of 5184 beads, 10 steps
    python -m paper_2512_13267_gb300.profile_cases mlp     # closure training + inference, B = 4096
    python -m paper_2512_13267_gb300.profile_cases sph     # cylinder cell, 16 384 fluid particles

Each case builds its inputs with the seeded generators of `synth`, runs a
few warm-up launches and then the launches a profiler captures, and exits 0.
"""
import sys

import numpy as np


def micro(boxes=304, edge=12.0, steps=10, calls=3):
    import torch
    from . import lhmm, synth
    batch = synth.make_batch(np.full(boxes, edge),
                             synth.random_velocity_gradients(boxes, seed=2), 2, flow="afbc")
    m = lhmm.Micro.from_batch(lhmm.dpd_params(flow="afbc", seed=2), batch)
    L = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((boxes, 6), dtype=torch.float64, device="cuda")
    for _ in range(calls):
        m.advance(L, steps, st)
    torch.cuda.synchronize()
    m.close()


def mlp(rows=4096, steps=4):
    import torch
    from . import lhmm
    c = lhmm.Closure(members=5, in_dim=67, hidden=256, n_hidden=4, out_dim=3, seed=1)
    c.set_normalization(np.zeros(67), np.ones(67), np.ones(3))
    rng = np.random.default_rng(0)
    X = torch.from_numpy(rng.normal(size=(65536, 67)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.normal(size=(65536, 3)).astype(np.float32)).cuda()
    for _ in range(steps):
        rws = torch.from_numpy(rng.integers(0, 65536, size=(5, rows)).astype(np.int32)).cuda()
        c.train_step(X, T, rows, lr=1e-3, weight_decay=1e-4, rows_dev=rws)
    mean = torch.zeros((16384, 3), dtype=torch.float32, device="cuda")
    spread = torch.zeros(16384, dtype=torch.float32, device="cuda")
    c.infer(X[:16384], mean, spread)
    torch.cuda.synchronize()
    c.close()


def sph(n_fluid=16384, cell=16.0, substeps=20):
    import torch
    from . import lhmm, synth
    pos, is_wall, L, dh = synth.cylinder_array(n_fluid_target=n_fluid, radius_frac=0.25, cell=cell)
    n, n_wall = pos.shape[0], int(is_wall.sum())
    p = lhmm.sph_params(n, n_wall, Lx=L, Ly=L, h=3 * dh, mass=dh * dh, rho0=1.0, c=2.5,
                        theta_pb=0.1, eta_s=0.1, dt=0.2 * dh / 2.5, body_force=(1e-3, 0.0))
    s = lhmm.Sph(p, pos, np.zeros_like(pos))
    Lout = torch.zeros((n_fluid, 9), dtype=torch.float32, device="cuda")
    for _ in range(3):
        s.step(substeps, L_out_dev=Lout)
    torch.cuda.synchronize()
    s.close()


if __name__ == "__main__":
    {"micro": micro, "mlp": mlp, "sph": sph}[sys.argv[1]]()
