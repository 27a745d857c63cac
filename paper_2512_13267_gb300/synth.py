"""Seeded synthetic inputs for the LHMM micro/macro hot path.

This module only makes inputs: initial bead states, box batches, velocity
gradients, SPH particle layouts.  It holds none of the method's arithmetic
(no forces, no integrator, no stress) and imports neither the CUDA library
nor the CPU oracle, so both sides consume identical inputs.

Workload shapes (sizes, compositions, distributions) follow the paper's
micro-domains and benchmark flows, restated in 3D periodic boxes:
  * one 10^3 box of 3000 beads under Lees-Edwards shear (virtual rheometer);
  * 1024 boxes with edges uniform in {6..12} (648..5184 beads), 20 % of the
    beads in N_d = 10 FENE chains, each box with its own velocity gradient
    (shear rate log-uniform in [1e-3, 1], 30 % planar extension);
  * the reverse-Poiseuille SPH channel of Sec. 6.1 and a periodic array of
    cylinders (Sec. 6.2) as SPH particle layouts.
"""
from dataclasses import dataclass, field

import numpy as np

# DPD/FENE parameter set of the 3D workloads (reduced units m = rc = kBT = 1)
DPD_PARAMS = dict(a_ij=25.0, gamma=4.5, sigma=3.0, kBT=1.0, rc=1.0, H_fene=30.0, R0=1.5,
                  dt=0.01, mass=1.0)
# Table 1 of the paper (2D melts): kept for the paper-faithful variant
DPD_PARAMS_PAPER_2D = dict(a_ij=25.0, gamma=4.5, sigma=3.0, kBT=1.0, rc=1.0, H_fene=50.0,
                           R0=1.5, dt=0.005, mass=1.0)
AFBC_CORE_FRAC = 24.0 / 76.0   # Table 2: l_core / l_total
AFBC_BC_FRAC = 13.0 / 76.0     # Table 2: l_bc / l_total
DENSITY = 3.0
DENSITY_PAPER_2D = 4.0  # Table 1: n_DPD (per area), dx = n^(-1/2) = 0.5
CHAIN_LEN = 10
POLYMER_FRACTION = 0.2


def n_chains_for(n_beads, chain_len=CHAIN_LEN, fraction=POLYMER_FRACTION):
    return int(round(fraction * n_beads / chain_len))


def serpentine_sites(n_side):
    """Lattice sites (ix, iy, iz) in boustrophedon order: consecutive sites are
    lattice neighbours, so consecutive beads of a chain start one spacing apart."""
    sites = []
    for iz in range(n_side):
        ys = range(n_side) if iz % 2 == 0 else range(n_side - 1, -1, -1)
        for row, iy in enumerate(ys):
            flip = (iz * n_side + row) % 2
            xs = range(n_side) if not flip else range(n_side - 1, -1, -1)
            for ix in xs:
                sites.append((ix, iy, iz))
    return np.asarray(sites, dtype=np.int64)


def serpentine_sites_2d(n_side):
    """Square-lattice sites (ix, iy, 0) in boustrophedon order."""
    sites = []
    for iy in range(n_side):
        xs = range(n_side) if iy % 2 == 0 else range(n_side - 1, -1, -1)
        for ix in xs:
            sites.append((ix, iy, 0))
    return np.asarray(sites, dtype=np.int64)


_SITE_CACHE = {}


def initial_box_state(edge, n_beads, seed, box_id=0, kBT=1.0, mass=1.0, L=None,
                      flow="afbc", jitter=0.1, dim=3):
    """Initial positions (in [0, edge)) and velocities, float32, shape (n, 3).

    Beads sit on the first n_beads sites of a serpentine cubic lattice of
    ceil(n^(1/3)) sites per side (square lattice of ceil(n^(1/2)) per side,
    z = 0, for dim = 2) with uniform jitter of +-jitter spacing; velocities
    are Maxwellian at kBT in each moving axis with the box mean removed, plus
    the imposed streaming profile (u = L r' about the box centre for AFBC,
    u_x = L_xy (y - Ly/2) for Lees-Edwards)."""
    edge = np.broadcast_to(np.asarray(edge, dtype=np.float64), (3,))
    if n_beads == 0:
        return np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32)
    rng = np.random.default_rng([int(seed), int(box_id), 0x5EED])
    root = 2.0 if dim == 2 else 3.0
    n_side = int(np.ceil(n_beads ** (1.0 / root) - 1e-9))
    while n_side ** int(root) < n_beads:
        n_side += 1
    key = (n_side, dim)
    if key not in _SITE_CACHE:
        _SITE_CACHE[key] = serpentine_sites_2d(n_side) if dim == 2 else serpentine_sites(n_side)
    sites = _SITE_CACHE[key][:n_beads]
    spacing = edge / n_side
    pos = (sites + 0.5) * spacing + rng.uniform(-jitter, jitter, size=(n_beads, 3)) * spacing
    pos = np.mod(pos, edge)
    vel = rng.normal(0.0, np.sqrt(kBT / mass), size=(n_beads, 3))
    if dim == 2:
        pos[:, 2] = 0.0
        vel[:, 2] = 0.0
    vel -= vel.mean(axis=0, keepdims=True)
    if L is not None:
        L = np.asarray(L, dtype=np.float64).reshape(3, 3)
        if flow == "afbc":
            vel += (pos - 0.5 * edge) @ L.T
        elif flow == "lees_edwards":
            vel[:, 0] += L[0, 1] * (pos[:, 1] - 0.5 * edge[1])
    pos32 = pos.astype(np.float32)
    # float32 rounding may land exactly on the upper edge: pull it inside
    for a in range(3):
        e32 = np.float32(edge[a])
        bad = pos32[:, a] >= e32
        pos32[bad, a] = np.nextafter(e32, np.float32(0))
    return pos32, vel.astype(np.float32)


@dataclass
class BoxBatch:
    """A batch of cubic boxes in one flat bead array (box b owns beads
    offsets[b] .. offsets[b+1])."""
    edges: np.ndarray            # (B, 3) float32
    n_beads: np.ndarray          # (B,) int32
    n_chains: np.ndarray         # (B,) int32
    chain_len: int
    L: np.ndarray                # (B, 9) float32, L_ab = du_a/dx_b
    pos: np.ndarray = field(default=None)   # (N, 3) float32
    vel: np.ndarray = field(default=None)   # (N, 3) float32
    flow: str = "afbc"
    seed: int = 0
    dim: int = 3

    @property
    def offsets(self):
        return np.concatenate([[0], np.cumsum(self.n_beads.astype(np.int64))])

    @property
    def n_boxes(self):
        return int(self.n_beads.shape[0])

    @property
    def total_beads(self):
        return int(self.n_beads.sum())

    def box_slice(self, b):
        o = self.offsets
        return slice(int(o[b]), int(o[b + 1]))

    def boxes(self, lo, hi):
        """The sub-batch of boxes lo .. hi-1 (one rank's share)."""
        o = self.offsets
        beads = slice(int(o[lo]), int(o[hi]))
        return BoxBatch(self.edges[lo:hi].copy(), self.n_beads[lo:hi].copy(),
                        self.n_chains[lo:hi].copy(), self.chain_len, self.L[lo:hi].copy(),
                        None if self.pos is None else self.pos[beads].copy(),
                        None if self.vel is None else self.vel[beads].copy(),
                        self.flow, self.seed, self.dim)


def make_batch(edges, L, seed, flow="afbc", chain_len=CHAIN_LEN, fraction=POLYMER_FRACTION,
               density=DENSITY, n_beads=None, kBT=1.0, with_state=True, dim=3):
    """A batch of boxes with per-box gradients L (B x 9).  dim = 2: square
    boxes in the x-y plane (z edge 1, unused), density per area."""
    edges = np.asarray(edges, dtype=np.float64)
    if edges.ndim == 1:
        edges = np.repeat(edges[:, None], 3, axis=1)
    if dim == 2:
        edges = edges.copy()
        edges[:, 2] = 1.0
    B = edges.shape[0]
    if n_beads is None:
        n_beads = np.rint(density * np.prod(edges, axis=1)).astype(np.int32)
    n_beads = np.asarray(n_beads, dtype=np.int32)
    n_chains = np.asarray([n_chains_for(int(n), chain_len, fraction) for n in n_beads],
                          dtype=np.int32)
    L = np.asarray(L, dtype=np.float32).reshape(B, 9)
    batch = BoxBatch(edges.astype(np.float32), n_beads, n_chains, chain_len, L, flow=flow,
                     seed=seed, dim=dim)
    if with_state:
        pos = np.empty((batch.total_beads, 3), np.float32)
        vel = np.empty((batch.total_beads, 3), np.float32)
        for b in range(B):
            sl = batch.box_slice(b)
            p, v = initial_box_state(edges[b], int(n_beads[b]), seed, b, kBT=kBT, L=L[b],
                                     flow=flow, dim=dim)
            pos[sl] = p
            vel[sl] = v
        batch.pos, batch.vel = pos, vel
    return batch


def random_velocity_gradients(n, seed, rate_range=(1e-3, 1.0), extension_fraction=0.3):
    """Per-box L (n, 9): shear rate log-uniform in rate_range; a fraction of
    boxes get planar extension diag(e, -e, 0), the rest simple shear L_xy."""
    rng = np.random.default_rng([int(seed), 0x6EAD])
    lo, hi = np.log10(rate_range[0]), np.log10(rate_range[1])
    rates = 10.0 ** rng.uniform(lo, hi, size=n)
    ext = rng.random(n) < extension_fraction
    L = np.zeros((n, 9), np.float32)
    L[~ext, 1] = rates[~ext]
    L[ext, 0] = rates[ext]
    L[ext, 4] = -rates[ext]
    return L


def batched_microsolver(n_boxes=1024, seed=2, edge_range=(6, 12), with_state=True):
    """The batched plain micro step: n_boxes AFBC boxes, edge ~ U{6..12}."""
    rng = np.random.default_rng([int(seed), 0xB0C5])
    edges = rng.integers(edge_range[0], edge_range[1] + 1, size=n_boxes).astype(np.float64)
    L = random_velocity_gradients(n_boxes, seed)
    return make_batch(edges, L, seed, flow="afbc", with_state=with_state)


def single_shear_box(seed=1, edge=10.0, shear_rate=0.1, n_beads=3000, n_chains=100):
    """One periodic box under Lees-Edwards shear du_x/dy = shear_rate."""
    L = np.zeros((1, 9), np.float32)
    L[0, 1] = shear_rate
    b = make_batch(np.asarray([edge]), L, seed, flow="lees_edwards",
                   n_beads=np.asarray([n_beads]), with_state=False)
    b.n_chains = np.asarray([n_chains], np.int32)
    p, v = initial_box_state(np.full(3, edge), n_beads, seed, 0, L=L[0], flow="lees_edwards")
    b.pos, b.vel = p, v
    return b


# ------------------------------------------------------------------ SPH layouts
def sph_lattice(nx, ny, Lx, Ly, seed=0, jitter=0.0):
    """nx x ny particles on a cell-centred lattice of the periodic box."""
    rng = np.random.default_rng([int(seed), 0x5A4])
    dx, dy = Lx / nx, Ly / ny
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    pos = np.stack([(ix.ravel() + 0.5) * dx, (iy.ravel() + 0.5) * dy], axis=1)
    if jitter > 0:
        pos += rng.uniform(-jitter, jitter, size=pos.shape) * np.array([dx, dy])
        pos = np.mod(pos, [Lx, Ly])
    return pos


def reverse_poiseuille_channel(nx=64, ny=32, Ly=4.0):
    """Sec. 6.1 channel: Lx = 2 Ly here so that nx x ny particles keep a square
    spacing dh = Ly / ny."""
    dh = Ly / ny
    Lx = nx * dh
    pos = sph_lattice(nx, ny, Lx, Ly)
    return pos, Lx, Ly, dh


def cylinder_array(n_fluid_target=16384, radius_frac=0.25, wall_layers=None, h_over_dh=3.0,
                   cell=1.0):
    """Periodic cell of width `cell` with one cylinder of radius radius_frac *
    cell (Sec. 6.2 geometry).  Returns (pos, is_wall, L, dh): lattice particles
    outside the cylinder are fluid (exactly n_fluid_target, first); those
    inside within h of its surface are fixed wall particles (last); the rest of
    the cylinder is empty."""
    area_frac = 1.0 - np.pi * radius_frac ** 2
    n_side = int(np.ceil(np.sqrt(n_fluid_target / area_frac)))
    while True:
        L = float(cell)
        dh = L / n_side
        pos = sph_lattice(n_side, n_side, L, L)
        r = np.hypot(pos[:, 0] - 0.5 * L, pos[:, 1] - 0.5 * L)
        R = radius_frac * L
        fluid = r >= R
        if fluid.sum() >= n_fluid_target:
            break
        n_side += 1
    h = h_over_dh * dh
    wall = (~fluid) & (r >= R - h)
    keep_fluid = np.flatnonzero(fluid)[:n_fluid_target]
    walls = np.flatnonzero(wall)
    pos = np.concatenate([pos[keep_fluid], pos[walls]], axis=0)
    is_wall = np.concatenate([np.zeros(len(keep_fluid), np.int32), np.ones(len(walls), np.int32)])
    return pos, is_wall, L, dh


def random_porous_medium(Ly=4.0, aspect=3.0, dh=1.0 / 16.0, n_obstacles=17, porosity=0.792,
                         mean_radius=0.425, h_over_dh=4.0, seed=7):
    """Synthetic stand-in for the paper's random porous medium (Sec. 6.3): a
    periodic Lx x Ly box (Lx = aspect Ly) with n_obstacles non-overlapping
    cylinders whose radii scatter by +-25 % around mean_radius, scaled so the
    solid area gives the stated porosity (the paper's obstacle table is not
    available).  Lattice particles of spacing dh outside the cylinders are
    fluid (first); those inside within h = h_over_dh dh of a surface are
    fixed wall particles (last).  Returns (pos, is_wall, Lx, Ly, dh, centres,
    radii)."""
    rng = np.random.default_rng([int(seed), 0x2A9])
    Lx = aspect * Ly
    r = mean_radius * (1.0 + 0.25 * rng.uniform(-1.0, 1.0, size=n_obstacles))
    r *= np.sqrt((1.0 - porosity) * Lx * Ly / (np.pi * np.sum(r ** 2)))
    centres = np.zeros((n_obstacles, 2))
    order = np.argsort(-r)  # place the largest first
    placed = []
    for k in order:
        for _ in range(100000):
            c = rng.uniform([0.0, 0.0], [Lx, Ly])
            ok = True
            for j in placed:
                d = c - centres[j]
                d -= np.array([Lx, Ly]) * np.rint(d / np.array([Lx, Ly]))
                if np.hypot(*d) < r[k] + r[j] + 2.0 * dh:
                    ok = False
                    break
            if ok:
                centres[k] = c
                placed.append(k)
                break
        else:
            raise RuntimeError("could not place the obstacles")
    nx, ny = int(round(Lx / dh)), int(round(Ly / dh))
    pos = sph_lattice(nx, ny, Lx, Ly)
    depth = np.full(pos.shape[0], -np.inf)  # how far inside the nearest cylinder
    for c, R in zip(centres, r):
        d = pos - c
        d -= np.array([Lx, Ly]) * np.rint(d / np.array([Lx, Ly]))
        depth = np.maximum(depth, R - np.hypot(d[:, 0], d[:, 1]))
    fluid = depth <= 0.0
    wall = (~fluid) & (depth <= h_over_dh * dh)
    pos = np.concatenate([pos[fluid], pos[wall]], axis=0)
    is_wall = np.concatenate([np.zeros(int(fluid.sum()), np.int32),
                              np.ones(int(wall.sum()), np.int32)])
    return pos, is_wall, Lx, Ly, dh, centres, r


def coupled_channel(nx=64, ny=32, Ly=4.0, box_beads=1500, seed=3, c_factor=10.0, U_o=0.25,
                    eta_s=0.1, eta_tot=None, delta_t=0.5):
    """The coupled reverse-Poiseuille workload: an nx x ny SPH channel of height
    Ly (square spacing dh = Ly/ny, Lx = nx dh), Wendland support h = 3 dh, one
    AFBC box of box_beads beads (density 3, 20 % in N_d = 10 chains) per
    particle.  The body force makes the Newtonian mean speed U_o for the total
    viscosity eta_tot (U_o = F rho Ly^2 / (48 eta)); the sound speed is
    c_factor U_o.  The SPH substeps per exchange interval delta_t follow the
    CFL rule of Appendix C evaluated with the particle spacing dh as length.
    Returns a dict of SPH settings and the box batch."""
    pos, Lx, Ly, dh = reverse_poiseuille_channel(nx, ny, Ly)
    n = pos.shape[0]
    eta_tot = eta_s + 0.01 if eta_tot is None else eta_tot
    F = 48.0 * eta_tot * U_o / Ly ** 2
    c = c_factor * U_o
    dt_cfl = 0.25 * min(dh / (1.5 * U_o + c), np.sqrt(dh / F), dh * dh / (2.0 * eta_tot))
    M = int(np.ceil(delta_t / dt_cfl))
    edge = (box_beads / DENSITY) ** (1.0 / 3.0)
    batch = make_batch(np.full(n, edge), np.zeros((n, 9), np.float32), seed, flow="afbc",
                       n_beads=np.full(n, box_beads))
    sph = dict(pos=pos, vel=np.zeros_like(pos), Lx=Lx, Ly=Ly, dh=dh, h=3.0 * dh,
               mass=dh * dh, rho0=1.0, c=c, eta_s=eta_s, body_force=F, substeps=M,
               dt=delta_t / M)
    return sph, batch


def melt_rheometer_batch(chain_len, shear_rates, replicas, edge=20.0, seed=11,
                         density=DENSITY_PAPER_2D):
    """2D polymer melts of the paper's micro model (Table 1: number density 4,
    all beads in chains of chain_len) in square periodic boxes under
    Lees-Edwards shear: `replicas` boxes per shear rate, box b sheared at
    shear_rates[b // replicas] (L_xy)."""
    rates = np.repeat(np.asarray(shear_rates, dtype=np.float64), int(replicas))
    B = rates.shape[0]
    L = np.zeros((B, 9), np.float32)
    L[:, 1] = rates
    n = int(round(density * edge * edge))
    n -= n % chain_len
    return make_batch(np.full(B, edge), L, seed, flow="lees_edwards", chain_len=chain_len,
                      fraction=1.0, n_beads=np.full(B, n), dim=2)
