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
