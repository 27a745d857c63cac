"""Multi-rank host path on CPU: box partition and the per-macro-step stress
all-gather, world size 2 over gloo, with the FP64 oracle standing in for
each rank's micro engine."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle as O
from paper_2512_13267_gb300 import sharding, synth as S


def test_partition_is_contiguous_and_balanced():
    rng = np.random.default_rng(0)
    n = rng.integers(648, 5185, size=1024)
    for world in (1, 2, 3, 8):
        r = sharding.partition_boxes(n, world)
        assert r[0][0] == 0 and r[-1][1] == 1024
        assert all(a[1] == b[0] for a, b in zip(r[:-1], r[1:]))
        loads = np.array([n[lo:hi].sum() for lo, hi in r])
        assert loads.max() - loads.min() <= 2 * n.max()
    assert sharding.partition_boxes([5, 5], 4)[-1][1] == 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    return S.make_batch(np.array([3.0, 4.0, 3.0, 5.0, 4.0]),
                        S.random_velocity_gradients(5, 4, rate_range=(0.05, 0.5)), 4)


def _advance(batch, ids, n_steps=3):
    par = O.dpd_params(flow_mode=O.FLOW_AFBC, seed=4)
    out = []
    for b in ids:
        sl = batch.box_slice(b)
        ob = O.Box(batch.edges[b], batch.pos[sl], batch.vel[sl], int(batch.n_chains[b]),
                   batch.chain_len, box_id=b)
        O.compute_forces(par, ob, batch.L[b])
        m, _, _ = O.advance(par, ob, batch.L[b], n_steps)
        out.append(m)
    return np.asarray(out)


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    batch = _batch()
    ranges = sharding.partition_boxes(batch.n_beads, world)
    lo, hi = ranges[rank]
    local = torch.from_numpy(_advance(batch, range(lo, hi)))
    full = sharding.gather_stress(local, ranges)
    t = torch.tensor([float(hi - lo)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)  # max-over-ranks reduction of the bench
    if rank == 0:
        q.put((full.numpy(), float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_reproduce_single_process_stress():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    full, tmax = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = _advance(_batch(), range(5))
    assert np.array_equal(full, ref)
    assert tmax >= 2


# ---------------------------------------------------------------- sharded coupled step
# The scheduling and exchange of sharding.ShardedCoupled with the FP64
# oracle standing in for the GPU SPH and micro engines: a small reverse-
# Poiseuille system (8 x 8 SPH particles, one 81-bead AFBC box each), two
# macro steps.  Two gloo ranks must reproduce the one-process run bit for
# bit, and their SPH replicas must stay identical.
N_SIDE, K_MICRO, M_SUB = 8, 3, 4


class _OracleSph:
    def __init__(self):
        n = N_SIDE * N_SIDE
        self.p = O.sph_params(n=n, Lx=1.0, Ly=1.0, h=3.0 / N_SIDE, mass=1.0 / n, rho0=1.0, c=1.0,
                              eta_s=0.1, dt=2e-3, body_force=(0.5, 0.0),
                              body_mode=O.BODY_REVERSE_POISEUILLE)
        self.pos = S.sph_lattice(N_SIDE, N_SIDE, 1.0, 1.0, seed=1, jitter=0.1).astype(np.float64)
        self.vel = np.zeros_like(self.pos)
        self.acc, _ = O.sph_accel(self.p, self.pos, self.vel)

    def step(self, stress):
        import torch
        s = stress.numpy()
        s3 = np.ascontiguousarray(np.stack([s[:, 0], s[:, 3], s[:, 1]], axis=1))
        O.sph_steps(self.p, self.pos, self.vel, self.acc, M_SUB, None, s3)
        _, d = O.sph_accel(self.p, self.pos, self.vel, stress3=s3)
        L4 = O.sph_velgrad(self.p, self.pos, self.vel, d)
        L = np.zeros((L4.shape[0], 9))
        L[:, 0], L[:, 1], L[:, 3], L[:, 4] = L4[:, 0], L4[:, 1], L4[:, 2], L4[:, 3]
        return torch.from_numpy(L)


class _OracleMicro:
    def __init__(self, lo, hi):
        self.par = O.dpd_params(flow_mode=O.FLOW_AFBC, seed=6, alpha=0.05)
        batch = S.make_batch(np.full(N_SIDE * N_SIDE, 3.0), np.zeros((N_SIDE * N_SIDE, 9)), 6)
        self.boxes = []
        for b in range(lo, hi):  # global box ids key the noise
            sl = batch.box_slice(b)
            ob = O.Box(batch.edges[b], batch.pos[sl], batch.vel[sl], int(batch.n_chains[b]),
                       batch.chain_len, box_id=b)
            O.compute_forces(self.par, ob, np.zeros(9))
            self.boxes.append(ob)

    def advance(self, L_local):
        import torch
        L = L_local.numpy()
        out = [O.advance(self.par, ob, L[i], K_MICRO)[0] for i, ob in enumerate(self.boxes)]
        return torch.from_numpy(np.asarray(out).reshape(-1, 6))


def _coupled(ranges, rank):
    import torch
    lo, hi = ranges[rank]
    sph = _OracleSph()
    c = sharding.ShardedCoupled(sph, _OracleMicro(lo, hi), ranges,
                                torch.zeros((N_SIDE * N_SIDE, 6), dtype=torch.float64))
    stress = c.step(2).numpy().copy()
    return stress, sph.pos.copy()


def _coupled_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n_beads = np.full(N_SIDE * N_SIDE, 81)
    stress, pos = _coupled(sharding.partition_boxes(n_beads, world), rank)
    q.put((rank, stress, pos))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_coupled_step_two_ranks_equal_one_process():
    ref_stress, ref_pos = _coupled([(0, N_SIDE * N_SIDE)], 0)
    assert np.abs(ref_stress).max() > 0
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_coupled_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict((r, (s, x)) for r, s, x in (q.get(timeout=300) for _ in range(2)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert np.array_equal(got[r][0], ref_stress)  # every rank holds the full stress
        assert np.array_equal(got[r][1], ref_pos)     # identical SPH replicas


def test_one_process_sharded_coupled_rejects_several_ranges():
    import torch
    with pytest.raises(ValueError):
        sharding.ShardedCoupled(None, None, [(0, 2), (2, 4)], torch.zeros((4, 6)))
