"""Box sharding across ranks (one process per GPU).

The micro-domains are independent, so the batch splits by box with no
data-path collective inside a micro step: each rank owns a contiguous,
size-balanced range of boxes.  Per macro step the only exchange is the SPH
side: the SPH step needs every box's stress (an all-gather of n x 6
doubles), and with the SPH particles replicated on every rank each rank
already holds the velocity gradients of its boxes.  ShardedCoupled drives
one coupled system this way.
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


class ShardedCoupled:
    """One coupled LHMM system spread over the ranks of a process group, one
    GPU per rank (coupling protocol Steps 1-4 with the micro step sharded).

    The SPH particles are replicated on every rank: the SPH kernels are
    bit-reproducible, so replicas fed the same stresses stay identical and
    need no broadcast.  The micro boxes are split into contiguous,
    bead-balanced ranges (partition_boxes); rank r advances boxes
    ranges[r] under its slice of the velocity gradients.  Per macro step the
    ranks all-gather the n x 6 stresses, the method's only exchange.

    sph:   replicated macroscale with step(stress_full) -> L_full, the SPH
           substeps of one exchange interval under the given polymer stress
           followed by the velocity gradients (n x 9) of the fluid particles
    micro: this rank's boxes, with advance(L_local) -> stress_local, the k'
           DPD steps of the interval and the (hi - lo) x 6 time-averaged
           stresses
    stress0: the n x 6 polymer stress the first macro step uses
    Without an initialised process group it runs the whole system in one
    process (ranges must then hold one range)."""

    def __init__(self, sph, micro, ranges, stress0, group=None):
        import torch.distributed as dist
        self.sph, self.micro, self.ranges, self.group = sph, micro, ranges, group
        self.distributed = dist.is_available() and dist.is_initialized()
        self.rank = dist.get_rank(group) if self.distributed else 0
        if not self.distributed and len(ranges) != 1:
            raise ValueError("without a process group the system runs as one range")
        self.stress = stress0

    def step(self, n_macro=1):
        """n_macro macro steps; returns the gathered n x 6 stress."""
        lo, hi = self.ranges[self.rank]
        for _ in range(n_macro):
            L = self.sph.step(self.stress)
            local = self.micro.advance(L[lo:hi])
            self.stress = (gather_stress(local, self.ranges, self.group) if self.distributed
                           else local)
        return self.stress


class GpuSph:
    """lhmm.Sph as the replicated macroscale of ShardedCoupled: `substeps`
    velocity-Verlet SPH steps per interval, then the gradients."""

    def __init__(self, sph, n_fluid, substeps):
        import torch
        self.sph, self.substeps = sph, int(substeps)
        self.L = torch.zeros((n_fluid, 9), dtype=torch.float32, device="cuda")

    def step(self, stress):
        self.sph.step(self.substeps, stress_dev=stress, L_out_dev=self.L)
        return self.L


class GpuMicro:
    """An lhmm.Micro holding one rank's boxes (created with box_id_offset =
    the range's first box, so its noise is the whole system's) as the
    sharded micro step of ShardedCoupled: k' DPD steps per interval."""

    def __init__(self, micro, micro_steps):
        import torch
        self.micro, self.k = micro, int(micro_steps)
        self.stress = torch.zeros((micro.n_boxes, 6), dtype=torch.float64, device="cuda")

    def advance(self, L_local):
        self.micro.advance(L_local.contiguous(), self.k, self.stress)
        return self.stress
