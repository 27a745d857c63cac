"""Box sharding across ranks (one process per GPU).

The micro-domains are independent, so the batch splits by box with no
data-path collective inside a macro step: each rank owns a contiguous,
size-balanced range of boxes.  Per macro step the only exchange is the SPH
side: each rank needs the velocity gradients of its boxes (a scatter of
n x 9 floats) and the SPH step needs every box's stress (an all-gather of
n x 6 doubles), both on the host-free device path via torch.distributed.
"""
import numpy as np


def partition_boxes(n_beads, world):
    """Contiguous box ranges [lo, hi) per rank with near-equal bead counts
    (greedy cut of the prefix sum at k/world of the total)."""
    n_beads = np.asarray(n_beads, dtype=np.int64)
    n = n_beads.shape[0]
    if world < 1:
        raise ValueError("world must be >= 1")
    pref = np.concatenate([[0], np.cumsum(n_beads)])
    total = pref[-1]
    cuts = [0]
    for k in range(1, world):
        target = total * k / world
        c = int(np.searchsorted(pref, target, side="left"))
        c = min(max(c, cuts[-1]), n)
        cuts.append(c)
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def gather_stress(local_stress, ranges, group=None):
    """All-gather each rank's (hi - lo) x 6 stress rows into the full n x 6
    array in box order (torch tensors; any backend)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    width = max(hi - lo for lo, hi in ranges)
    pad = torch.zeros((width, local_stress.shape[1]), dtype=local_stress.dtype,
                      device=local_stress.device)
    pad[: local_stress.shape[0]] = local_stress
    parts = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([parts[r][: hi - lo] for r, (lo, hi) in enumerate(ranges)], dim=0)
