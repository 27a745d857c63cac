"""ctypes front end of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It never touches the CUDA library.
"""
import ctypes as C
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)
from build import build_oracle  # noqa: E402

FLOW_PERIODIC, FLOW_LEES_EDWARDS, FLOW_AFBC = 0, 1, 2
ERR_BOND_OVERSTRETCH, ERR_NAN, ERR_ARG = 1, 2, 4
KERNEL_WENDLAND_C2, KERNEL_LUCY = 0, 1
VISC_DERIVED_2D, VISC_PAPER_LITERAL = 0, 1
BODY_UNIFORM, BODY_REVERSE_POISEUILLE = 0, 1


class DpdParams(C.Structure):
    _fields_ = [
        ("a_ij", C.c_double), ("gamma", C.c_double), ("sigma", C.c_double),
        ("kBT", C.c_double), ("rc", C.c_double), ("H_fene", C.c_double),
        ("R0", C.c_double), ("dt", C.c_double), ("mass", C.c_double),
        ("seed", C.c_uint64), ("flow_mode", C.c_int),
        ("core_frac", C.c_double), ("bc_frac", C.c_double),
        ("dpd_on_bonded", C.c_int), ("alpha", C.c_double), ("lambda_star", C.c_double),
        ("dim", C.c_int), ("exclude_bonds", C.c_int), ("afbc_mode", C.c_int),
    ]


class _Box(C.Structure):
    _fields_ = [
        ("box_id", C.c_int), ("edge", C.c_double * 3), ("n", C.c_int),
        ("n_chains", C.c_int), ("chain_len", C.c_int),
        ("pos", C.POINTER(C.c_double)), ("vel", C.POINTER(C.c_double)),
        ("force", C.POINTER(C.c_double)), ("step", C.c_uint64), ("le_offset", C.c_double),
    ]


class SphParams(C.Structure):
    _fields_ = [
        ("n", C.c_int), ("Lx", C.c_double), ("Ly", C.c_double), ("h", C.c_double),
        ("mass", C.c_double), ("rho0", C.c_double), ("c", C.c_double),
        ("theta_pb", C.c_double), ("eta_s", C.c_double), ("zeta_s", C.c_double),
        ("dt", C.c_double), ("kernel", C.c_int), ("visc_coeffs", C.c_int),
        ("body_force", C.c_double * 2), ("body_mode", C.c_int),
    ]


_lib = None
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        L = C.CDLL(path)
        u32p = C.POINTER(C.c_uint32)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_pair_theta.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_uint64]
        L.orc_pair_theta.restype = C.c_double
        L.orc_theta_from_words.argtypes = [C.c_uint32, C.c_uint32]
        L.orc_theta_from_words.restype = C.c_double
        L.orc_compute_forces.argtypes = [C.POINTER(DpdParams), C.POINTER(_Box), _D, C.c_int, _D]
        L.orc_advance.argtypes = [C.POINTER(DpdParams), C.POINTER(_Box), _D, C.c_int, _D, _D]
        L.orc_advance_batch.argtypes = [C.POINTER(DpdParams), C.POINTER(_Box), C.c_int, _D,
                                        C.c_int, _D, _D, C.c_int, _I]
        L.orc_ik_sample.argtypes = [C.POINTER(DpdParams), C.POINTER(_Box), _D, _D]
        L.orc_diagnostics.argtypes = [C.POINTER(DpdParams), C.POINTER(_Box), _D, _D]
        L.orc_afbc_region.argtypes = [C.POINTER(DpdParams), _D, _D]
        L.orc_segment_fraction.argtypes = [_D, _D, _D]
        L.orc_segment_fraction.restype = C.c_double
        L.orc_max_threads.restype = C.c_int
        L.orc_sph_W.argtypes = [C.c_int, C.c_double, C.c_double]
        L.orc_sph_W.restype = C.c_double
        L.orc_sph_F.argtypes = [C.c_int, C.c_double, C.c_double]
        L.orc_sph_F.restype = C.c_double
        L.orc_sph_pressure.argtypes = [C.POINTER(SphParams), C.c_double]
        L.orc_sph_pressure.restype = C.c_double
        L.orc_sph_density.argtypes = [C.POINTER(SphParams), _D, _D]
        L.orc_sph_accel.argtypes = [C.POINTER(SphParams), _D, _D, _I, _D, _D, _D]
        L.orc_sph_velgrad.argtypes = [C.POINTER(SphParams), _D, _D, _D, _D]
        L.orc_sph_steps.argtypes = [C.POINTER(SphParams), _D, _D, _D, _I, _D, C.c_int]
        L.orc_mlp_n_params.argtypes = [C.c_int, _I]
        L.orc_mlp_n_params.restype = C.c_long
        L.orc_mlp_forward.argtypes = [C.c_int, _I, _D, C.c_int, _D, _D]
        L.orc_mlp_loss_grad.argtypes = [C.c_int, _I, _D, C.c_int, _D, _D, _D]
        L.orc_mlp_loss_grad.restype = C.c_double
        L.orc_adamw_step.argtypes = [C.c_long, _D, _D, _D, _D, C.c_double, C.c_double,
                                     C.c_double, C.c_double, C.c_double, C.c_long]
        L.orc_gelu.argtypes = [C.c_double]
        L.orc_gelu.restype = C.c_double
        _lib = L
    return _lib


def _dp(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _ip(a):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_I)


# ---------------------------------------------------------------- random numbers
def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def pair_theta(seed, box_id, i, j, step):
    return lib().orc_pair_theta(seed, box_id, i, j, step)


def theta_from_words(x0, x1):
    return lib().orc_theta_from_words(x0, x1)


# ---------------------------------------------------------------- micro
def dpd_params(**kw):
    """Build the parameter struct; keys follow orc_dpd_params."""
    defaults = dict(a_ij=25.0, gamma=4.5, sigma=3.0, kBT=1.0, rc=1.0, H_fene=30.0, R0=1.5,
                    dt=0.01, mass=1.0, seed=1, flow_mode=FLOW_PERIODIC,
                    core_frac=24.0 / 76.0, bc_frac=13.0 / 76.0, dpd_on_bonded=1,
                    alpha=1.0, lambda_star=1.0, dim=3, exclude_bonds=0, afbc_mode=0)
    defaults.update(kw)
    return DpdParams(**defaults)


class Box:
    """One micro-domain held in FP64 numpy arrays."""

    def __init__(self, edge, pos, vel, n_chains, chain_len, box_id=0, step=0, le_offset=0.0,
                 force=None):
        self.pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3).copy()
        self.vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(-1, 3).copy()
        n = self.pos.shape[0]
        self.force = (np.zeros((n, 3)) if force is None
                      else np.ascontiguousarray(force, dtype=np.float64).reshape(-1, 3).copy())
        e = np.broadcast_to(np.asarray(edge, dtype=np.float64), (3,))
        self.s = _Box(box_id, (C.c_double * 3)(*e), n, n_chains, chain_len,
                      _dp(self.pos), _dp(self.vel), _dp(self.force), step, le_offset)

    @property
    def step(self):
        return int(self.s.step)

    @property
    def le_offset(self):
        return float(self.s.le_offset)

    @property
    def n(self):
        return self.pos.shape[0]


def _L(L):
    L = np.ascontiguousarray(np.asarray(L, dtype=np.float64).reshape(9))
    return L


def compute_forces(p, box, L=None, brute=False):
    L = _L(np.zeros(9) if L is None else L)
    v6 = np.zeros(6)
    err = lib().orc_compute_forces(C.byref(p), C.byref(box.s), _dp(L), int(brute), _dp(v6))
    return box.force.copy(), v6, err


def advance(p, box, L, n_steps):
    L = _L(L)
    m = np.zeros(6)
    q = np.zeros(6)
    err = lib().orc_advance(C.byref(p), C.byref(box.s), _dp(L), int(n_steps), _dp(m), _dp(q))
    return m, q, err


def advance_batch(p, boxes, L, n_steps, n_threads=0):
    nb = len(boxes)
    arr = (_Box * nb)(*[b.s for b in boxes])
    L = np.ascontiguousarray(np.asarray(L, dtype=np.float64).reshape(nb, 9))
    m = np.zeros((nb, 6))
    q = np.zeros((nb, 6))
    st = np.zeros(nb, dtype=np.int32)
    err = lib().orc_advance_batch(C.byref(p), arr, nb, _dp(L), int(n_steps), _dp(m), _dp(q),
                                  int(n_threads), _ip(st))
    for k, b in enumerate(boxes):  # copy back scalars advanced in the array copy
        b.s.step = arr[k].step
        b.s.le_offset = arr[k].le_offset
    return m, q, st, err


def ik_sample(p, box, L=None):
    L = _L(np.zeros(9) if L is None else L)
    pi6 = np.zeros(6)
    err = lib().orc_ik_sample(C.byref(p), C.byref(box.s), _dp(L), _dp(pi6))
    return pi6, err


def diagnostics(p, box, L=None):
    """[P_x, P_y, P_z, kinetic, conservative DPD potential, FENE potential,
    total energy, 0] of one box, and the error bits."""
    L = _L(np.zeros(9) if L is None else L)
    out = np.zeros(8)
    err = lib().orc_diagnostics(C.byref(p), C.byref(box.s), _dp(L), _dp(out))
    return out, err


def afbc_region(p, edge, r):
    e = np.ascontiguousarray(np.broadcast_to(np.asarray(edge, np.float64), (3,)))
    r = np.ascontiguousarray(np.asarray(r, np.float64))
    return lib().orc_afbc_region(C.byref(p), _dp(e), _dp(r))


def segment_fraction(a, b, half):
    a, b, half = (np.ascontiguousarray(np.asarray(x, np.float64)) for x in (a, b, half))
    return lib().orc_segment_fraction(_dp(a), _dp(b), _dp(half))


def max_threads():
    return lib().orc_max_threads()


# ---------------------------------------------------------------- SPH
def sph_params(**kw):
    d = dict(n=0, Lx=1.0, Ly=1.0, h=0.3, mass=1.0, rho0=1.0, c=1.0, theta_pb=0.1,
             eta_s=0.1, zeta_s=0.0, dt=1e-3, kernel=KERNEL_WENDLAND_C2,
             visc_coeffs=VISC_DERIVED_2D, body_force=(0.0, 0.0), body_mode=BODY_UNIFORM)
    d.update(kw)
    bf = d.pop("body_force")
    p = SphParams(**d)
    p.body_force[0], p.body_force[1] = bf
    return p


def sph_W(kernel, r, h):
    return lib().orc_sph_W(kernel, r, h)


def sph_F(kernel, r, h):
    return lib().orc_sph_F(kernel, r, h)


def sph_pressure(p, rho):
    return lib().orc_sph_pressure(C.byref(p), rho)


def sph_density(p, pos):
    pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 2)
    d = np.zeros(pos.shape[0])
    lib().orc_sph_density(C.byref(p), _dp(pos), _dp(d))
    return d


def sph_accel(p, pos, vel, is_wall=None, stress3=None):
    pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 2)
    vel = np.ascontiguousarray(vel, np.float64).reshape(-1, 2)
    n = pos.shape[0]
    acc = np.zeros((n, 2))
    d = np.zeros(n)
    w = None if is_wall is None else np.ascontiguousarray(is_wall, np.int32)
    s = None if stress3 is None else np.ascontiguousarray(stress3, np.float64).reshape(-1, 3)
    lib().orc_sph_accel(C.byref(p), _dp(pos), _dp(vel), None if w is None else _ip(w),
                        None if s is None else _dp(s), _dp(acc), _dp(d))
    return acc, d


def sph_velgrad(p, pos, vel, d):
    pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 2)
    vel = np.ascontiguousarray(vel, np.float64).reshape(-1, 2)
    d = np.ascontiguousarray(d, np.float64)
    L4 = np.zeros((pos.shape[0], 4))
    lib().orc_sph_velgrad(C.byref(p), _dp(pos), _dp(vel), _dp(d), _dp(L4))
    return L4


def sph_steps(p, pos, vel, acc, n_sub, is_wall=None, stress3=None):
    """In place on pos, vel, acc (float64 C-contiguous)."""
    w = None if is_wall is None else np.ascontiguousarray(is_wall, np.int32)
    s = None if stress3 is None else np.ascontiguousarray(stress3, np.float64).reshape(-1, 3)
    lib().orc_sph_steps(C.byref(p), _dp(pos), _dp(vel), _dp(acc),
                        None if w is None else _ip(w), None if s is None else _dp(s), int(n_sub))


# ---------------------------------------------------------------- MLP
def mlp_n_params(dims):
    d = np.ascontiguousarray(dims, np.int32)
    return lib().orc_mlp_n_params(len(dims) - 1, _ip(d))


def mlp_forward(dims, params, x):
    d = np.ascontiguousarray(dims, np.int32)
    x = np.ascontiguousarray(x, np.float64)
    y = np.zeros((x.shape[0], dims[-1]))
    lib().orc_mlp_forward(len(dims) - 1, _ip(d), _dp(np.ascontiguousarray(params, np.float64)),
                          x.shape[0], _dp(x), _dp(y))
    return y


def mlp_loss_grad(dims, params, x, target):
    d = np.ascontiguousarray(dims, np.int32)
    params = np.ascontiguousarray(params, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    t = np.ascontiguousarray(target, np.float64)
    g = np.zeros_like(params)
    loss = lib().orc_mlp_loss_grad(len(dims) - 1, _ip(d), _dp(params), x.shape[0], _dp(x),
                                   _dp(t), _dp(g))
    return loss, g


def adamw_step(params, grad, m, v, lr, beta1, beta2, eps, wd, t):
    """In place on params, m, v (float64 C-contiguous)."""
    lib().orc_adamw_step(params.size, _dp(params), _dp(np.ascontiguousarray(grad, np.float64)),
                         _dp(m), _dp(v), lr, beta1, beta2, eps, wd, int(t))


def gelu(x):
    return lib().orc_gelu(float(x))
