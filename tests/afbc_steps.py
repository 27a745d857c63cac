"""One-step parity of the AFBC update along the GPU trajectory.

The BC shell makes a bead's velocity jump when it crosses a region boundary
(core / BC / buffer) and, with afbc_mode = 1, when it changes cell (the mean
it is measured against changes).  A FP32 and a FP64 trajectory of the same
box drift apart by ~1e-7, so over many steps one of them eventually meets
such a boundary a step before the other and the trajectories separate for
good.  That is a discrete decision taken on rounded inputs, not a wrong
update, so these tests restart the oracle from the GPU state before every
step (same positions, velocities, forces, step counter) and compare one step
at a time.  Beads of a cell that holds a bead within `eps` of a boundary
could be classified either way; their velocities are left out of that step's
comparison and counted (positions do not depend on the decision).
"""
import numpy as np

import oracle as O


def ambiguous_beads(pos, edge, dim, core_frac, bc_frac, rc=1.0, eps=1e-5):
    """Beads whose region or cell could flip under a rounding of eps, and
    every bead sharing a cell with one (whose mean then changes)."""
    d = 2 if dim == 2 else 3
    E = np.asarray(edge, np.float64)[:d]
    x = pos[:, :d]
    rp = np.abs(x - 0.5 * E)
    near = np.zeros(len(pos), bool)
    for h in (0.5 * core_frac * E, (0.5 * core_frac + bc_frac) * E):
        near |= (np.abs(rp - h) < eps).any(axis=1)
    nc = np.floor(E / rc).astype(int)
    wf = E / nc  # the oracle's cells; the kernel's FP32 width differs by ~1 ulp
    cidx = np.clip(np.floor(x / wf).astype(int), 0, nc - 1)
    frac = x / wf - np.floor(x / wf)
    near |= ((frac < eps) | (frac > 1 - eps)).any(axis=1)
    cell = np.ravel_multi_index(tuple(cidx.T), tuple(nc))
    bad_cells = set(cell[near].tolist())
    # a bead near a cell face may be binned in the neighbour too
    for i in np.where(near)[0]:
        for a in range(d):
            for s in (-1, 1):
                c = cidx[i].copy()
                c[a] = (c[a] + s) % nc[a]
                bad_cells.add(int(np.ravel_multi_index(tuple(c), tuple(nc))))
    return np.isin(cell, list(bad_cells))


def stepwise_afbc_parity(m, op, batch, n_steps, dim=3, vel_tol=1e-4, pos_tol=1e-5):
    """Advance the GPU one step at a time; before each step restart an
    oracle box from the GPU state and advance it one step too.  Returns the
    number of bead velocities left out as ambiguous."""
    import torch
    L = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    skipped = 0
    for _ in range(n_steps):
        before = [m.get_state(b) for b in range(batch.n_boxes)]
        m.advance(L, 1, st)
        m.sync()
        for b in range(batch.n_boxes):
            pos, vel, f, step, _ = before[b]
            ob = O.Box(batch.edges[b], pos, vel, int(batch.n_chains[b]), batch.chain_len,
                       box_id=b, step=step, force=f)
            _, _, err = O.advance(op, ob, batch.L[b], 1)
            assert err == 0
            gpos, gvel, _, gstep, _ = m.get_state(b)
            assert gstep == step + 1
            E = batch.edges[b][0]
            dp = gpos - ob.pos
            dp -= E * np.rint(dp / E)
            assert np.abs(dp).max() <= pos_tol, (b, step, np.abs(dp).max())
            amb = ambiguous_beads(ob.pos, batch.edges[b], dim, op.core_frac, op.bc_frac)
            dv = np.abs(gvel - ob.vel).max(axis=1)
            ok = dv <= vel_tol
            assert np.all(ok | amb), (b, step, np.where(~(ok | amb))[0], dv[~(ok | amb)])
            skipped += int(np.count_nonzero(amb & ~ok))
    return skipped
