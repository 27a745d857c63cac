"""Thin ctypes binding of the LHMM C ABI (include/lhmm.h).

Argument marshalling only: every step of the hot path runs in the CUDA
library.  Device buffers are torch CUDA tensors (their data_ptr is passed),
streams are torch.cuda.Stream objects or raw cudaStream_t integers.  If the
library is missing this module raises; there is no CPU fallback.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblhmm.so")

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_BOND_OVERSTRETCH, ERR_CELL_OVERFLOW, ERR_NAN, \
    ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_FORCE_RANGE = range(10)
BOX_BOND_OVERSTRETCH, BOX_NAN, BOX_CELL_OVERFLOW, BOX_FORCE_RANGE = 1, 2, 4, 8
FLOW_PERIODIC, FLOW_LEES_EDWARDS, FLOW_AFBC = 0, 1, 2
FLOWS = {"periodic": FLOW_PERIODIC, "lees_edwards": FLOW_LEES_EDWARDS, "afbc": FLOW_AFBC}


class LhmmError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


class DpdParams(C.Structure):
    _fields_ = [
        ("a_ij", C.c_float), ("gamma", C.c_float), ("sigma", C.c_float), ("kBT", C.c_float),
        ("rc", C.c_float), ("H_fene", C.c_float), ("R0", C.c_float), ("dt", C.c_float),
        ("mass", C.c_float), ("seed", C.c_uint64), ("flow_mode", C.c_int),
        ("afbc_core_frac", C.c_float), ("afbc_bc_frac", C.c_float), ("dpd_on_bonded", C.c_int),
        ("alpha", C.c_double), ("lambda_star", C.c_double), ("dim", C.c_int),
        ("exclude_bonds", C.c_int), ("afbc_mode", C.c_int),
    ]


class BatchDesc(C.Structure):
    _fields_ = [("n_boxes", C.c_int), ("box_edge", C.POINTER(C.c_float)),
                ("n_beads", C.POINTER(C.c_int)), ("n_chains", C.POINTER(C.c_int)),
                ("chain_len", C.c_int), ("box_id_offset", C.c_int)]


class SphParams(C.Structure):
    _fields_ = [
        ("n", C.c_int), ("n_wall", C.c_int), ("Lx", C.c_float), ("Ly", C.c_float),
        ("h", C.c_float), ("mass", C.c_float), ("rho0", C.c_float), ("c", C.c_float),
        ("theta_pb", C.c_float), ("eta_s", C.c_float), ("zeta_s", C.c_float), ("dt", C.c_float),
        ("kernel", C.c_int), ("visc_coeffs", C.c_int), ("body_force", C.c_float * 2),
        ("body_mode", C.c_int),
    ]


SPH_WENDLAND_C2, SPH_LUCY = 0, 1
SPH_VISC_DERIVED_2D, SPH_VISC_PAPER_LITERAL = 0, 1
SPH_BODY_UNIFORM, SPH_BODY_REVERSE_POISEUILLE = 0, 1

_lib = None
_F = C.POINTER(C.c_float)
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_U32 = C.POINTER(C.c_uint32)
_U64 = C.POINTER(C.c_uint64)


def lib():
    """Load liblhmm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.lhmm_status_string.argtypes = [C.c_int]
        L.lhmm_status_string.restype = C.c_char_p
        L.lhmm_micro_create.argtypes = [C.POINTER(DpdParams), C.POINTER(BatchDesc), _D, _F, _F,
                                        vp, C.POINTER(vp)]
        L.lhmm_micro_destroy.argtypes = [vp]
        L.lhmm_micro_advance.argtypes = [vp, vp, vp, C.c_int, C.c_int, vp, vp, vp]
        L.lhmm_micro_advance_host.argtypes = [vp, _F, C.c_int, _D, _D, vp]
        L.lhmm_micro_sync.argtypes = [vp, _U32]
        L.lhmm_micro_get_state.argtypes = [vp, C.c_int, _D, _F, _F, _U64, _F]
        L.lhmm_micro_set_state.argtypes = [vp, C.c_int, _D, _F, _F, C.c_uint64, C.c_float]
        L.lhmm_micro_info.argtypes = [vp, _I, C.POINTER(C.c_int64), _I]
        L.lhmm_micro_autotune.argtypes = [vp, vp, C.c_int, vp]
        L.lhmm_micro_diagnostics.argtypes = [vp, vp, vp]
        L.lhmm_micro_plan.argtypes = [vp, _I, C.c_int, _I, _I, _I, _I]
        L.lhmm_micro_set_variant.argtypes = [vp, C.c_int, C.c_int]
        L.lhmm_micro_set_list_variant.argtypes = [vp, C.c_int]
        L.lhmm_sph_create.argtypes = [C.POINTER(SphParams), _F, _F, vp, C.POINTER(vp)]
        L.lhmm_sph_destroy.argtypes = [vp]
        L.lhmm_sph_step.argtypes = [vp, vp, C.c_int, vp, vp]
        L.lhmm_sph_recompute_forces.argtypes = [vp, vp, vp]
        L.lhmm_sph_get_state.argtypes = [vp, _F, _F, _F, _F]
        L.lhmm_sph_velgrad_noalloc.argtypes = [C.POINTER(SphParams), vp, vp, vp, vp]
        L.lhmm_sph_info.argtypes = [vp, _I, _I]
        L.lhmm_coupled_create.argtypes = [vp, vp, C.c_int, C.c_int, C.POINTER(vp)]
        L.lhmm_coupled_destroy.argtypes = [vp]
        L.lhmm_coupled_step.argtypes = [vp, C.c_int, C.c_int, vp]
        L.lhmm_coupled_exchange.argtypes = [vp, C.POINTER(vp), C.POINTER(vp)]
        L.lhmm_coupled_copy_exchange.argtypes = [vp, _F, _D]
        L.lhmm_coupled_set_closure.argtypes = [vp, vp, C.c_float, C.c_float, C.c_int]
        L.lhmm_coupled_enable_gate.argtypes = [vp, C.c_int]
        L.lhmm_coupled_set_gate.argtypes = [vp, C.c_float, C.c_int, C.c_int, C.c_int]
        L.lhmm_coupled_set_online_calibration.argtypes = [vp, C.c_int, C.c_float, _F]
        L.lhmm_coupled_gate_stats.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                              C.POINTER(C.c_int64), _D, _D]
        L.lhmm_coupled_closure_inputs.argtypes = [vp, _F]
        L.lhmm_micro_advance_dev_count.argtypes = [vp, vp, vp, vp, C.c_int, C.c_int, vp, vp, vp]
        L.lhmm_closure_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64,
                                          C.POINTER(vp)]
        L.lhmm_closure_destroy.argtypes = [vp]
        L.lhmm_closure_set_normalization.argtypes = [vp, _F, _F, _F]
        L.lhmm_closure_train_step.argtypes = [vp, vp, vp, vp, C.c_int, C.c_float, C.c_float, vp, vp]
        L.lhmm_closure_infer.argtypes = [vp, vp, C.c_int, vp, vp, vp]
        L.lhmm_closure_forward.argtypes = [vp, vp, C.c_int, _F]
        L.lhmm_closure_get_params.argtypes = [vp, C.c_int, _F]
        L.lhmm_closure_set_params.argtypes = [vp, C.c_int, _F]
        L.lhmm_closure_get_grad.argtypes = [vp, C.c_int, _F]
        L.lhmm_closure_info.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.lhmm_closure_set_gemm.argtypes = [vp, C.c_int]
        L.lhmm_closure_sync.argtypes = [vp]
        _lib = L
    return _lib


def status_string(s):
    return lib().lhmm_status_string(int(s)).decode()


def check(status, where):
    if status != OK:
        raise LhmmError(status, where)


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _ptr(t):
    """Device pointer of a torch CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _np(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(C.POINTER(np.ctypeslib.as_ctypes_type(dtype)))


def dpd_params(flow="afbc", seed=1, alpha=1.0, lambda_star=1.0, dpd_on_bonded=1,
               afbc_core_frac=24.0 / 76.0, afbc_bc_frac=13.0 / 76.0, dim=3, exclude_bonds=0,
               afbc_mode=0, **phys):
    d = dict(a_ij=25.0, gamma=4.5, sigma=3.0, kBT=1.0, rc=1.0, H_fene=30.0, R0=1.5, dt=0.01,
             mass=1.0)
    d.update(phys)
    flow_mode = FLOWS[flow] if isinstance(flow, str) else int(flow)
    return DpdParams(seed=seed, flow_mode=flow_mode, afbc_core_frac=afbc_core_frac,
                     afbc_bc_frac=afbc_bc_frac, dpd_on_bonded=dpd_on_bonded, alpha=alpha,
                     lambda_star=lambda_star, dim=dim, exclude_bonds=exclude_bonds,
                     afbc_mode=afbc_mode, **d)


class Micro:
    """A batch of DPD/FENE micro-domains resident on the GPU (lhmm_micro_*)."""

    def __init__(self, params, edges, n_beads, n_chains, chain_len, pos0, vel0, L0=None,
                 stream=None, box_id_offset=0):
        L = lib()
        edges, pe = _np(np.asarray(edges, np.float32).reshape(-1, 3), np.float32)
        nb, pn = _np(n_beads, np.int32)
        nch, pc = _np(n_chains, np.int32)
        pos0, pp = _np(np.asarray(pos0, np.float64).reshape(-1, 3), np.float64)
        vel0, pv = _np(np.asarray(vel0, np.float32).reshape(-1, 3), np.float32)
        self.params = params
        self.n_boxes = int(nb.shape[0])
        self.n_beads = nb.copy()
        self.offsets = np.concatenate([[0], np.cumsum(nb.astype(np.int64))])
        pL = None
        if L0 is not None:
            L0, pL = _np(np.asarray(L0, np.float32).reshape(self.n_boxes, 9), np.float32)
        desc = BatchDesc(self.n_boxes, pe, pn, pc, int(chain_len), int(box_id_offset))
        h = C.c_void_p()
        check(L.lhmm_micro_create(C.byref(params), C.byref(desc), pp, pv, pL, _stream_ptr(stream),
                                  C.byref(h)), "lhmm_micro_create")
        self.h = h

    @classmethod
    def from_batch(cls, params, batch, stream=None, box_id_offset=0):
        return cls(params, batch.edges, batch.n_beads, batch.n_chains, batch.chain_len,
                   batch.pos, batch.vel, L0=batch.L, stream=stream, box_id_offset=box_id_offset)

    def close(self):
        if getattr(self, "h", None):
            lib().lhmm_micro_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def advance(self, L_dev, n_steps, stress_dev, stress_sq_dev=None, box_idx_dev=None,
                stream=None):
        n_active = self.n_boxes if box_idx_dev is None else int(box_idx_dev.numel())
        if box_idx_dev is not None and n_active == 0:
            return  # nothing to advance
        check(lib().lhmm_micro_advance(self.h, _ptr(L_dev), _ptr(box_idx_dev), n_active,
                                       int(n_steps), _ptr(stress_dev), _ptr(stress_sq_dev),
                                       _stream_ptr(stream)), "lhmm_micro_advance")

    def advance_host(self, L_host, n_steps, stress_host=None, stress_sq_host=None, stream=None):
        L_host, pL = _np(np.asarray(L_host, np.float32).reshape(self.n_boxes, 9), np.float32)
        if stress_host is None:
            stress_host = np.zeros((self.n_boxes, 6))
        ps = stress_host.ctypes.data_as(_D)
        pq = None if stress_sq_host is None else stress_sq_host.ctypes.data_as(_D)
        check(lib().lhmm_micro_advance_host(self.h, pL, int(n_steps), ps, pq,
                                            _stream_ptr(stream)), "lhmm_micro_advance_host")
        return stress_host

    def diagnostics(self, diag_dev, stream=None):
        """FP64 [P_x, P_y, P_z, kinetic, DPD potential, FENE potential, total
        energy, over-stretch flag] per box into diag_dev (n_boxes x 8)."""
        check(lib().lhmm_micro_diagnostics(self.h, _ptr(diag_dev), _stream_ptr(stream)),
              "lhmm_micro_diagnostics")

    def sync(self, raise_on_error=True):
        st = np.zeros(max(self.n_boxes, 1), np.uint32)
        s = lib().lhmm_micro_sync(self.h, st.ctypes.data_as(_U32))
        if raise_on_error:
            check(s, "lhmm_micro_sync")
        return s, st[: self.n_boxes]

    def get_state(self, box):
        n = int(self.n_beads[box])
        pos = np.zeros((n, 3), np.float64)
        vel = np.zeros((n, 3), np.float32)
        frc = np.zeros((n, 3), np.float32)
        step = C.c_uint64()
        le = C.c_float()
        check(lib().lhmm_micro_get_state(self.h, int(box), pos.ctypes.data_as(_D),
                                         vel.ctypes.data_as(_F), frc.ctypes.data_as(_F),
                                         C.byref(step), C.byref(le)), "lhmm_micro_get_state")
        return pos, vel, frc, int(step.value), float(le.value)

    def set_state(self, box, pos, vel, force, step, le_offset=0.0):
        pos, pp = _np(np.asarray(pos, np.float64).reshape(-1, 3), np.float64)
        vel, pv = _np(np.asarray(vel, np.float32).reshape(-1, 3), np.float32)
        force, pf = _np(np.asarray(force, np.float32).reshape(-1, 3), np.float32)
        check(lib().lhmm_micro_set_state(self.h, int(box), pp, pv, pf, int(step),
                                         float(le_offset)), "lhmm_micro_set_state")

    def autotune(self, L_dev, probe_steps=10, stream=None):
        check(lib().lhmm_micro_autotune(self.h, _ptr(L_dev), int(probe_steps),
                                        _stream_ptr(stream)), "lhmm_micro_autotune")

    def plan(self):
        n = C.c_int()
        check(lib().lhmm_micro_plan(self.h, C.byref(n), 0, None, None, None, None),
              "lhmm_micro_plan")
        k = n.value
        arrs = [np.zeros(max(k, 1), np.int32) for _ in range(4)]
        check(lib().lhmm_micro_plan(self.h, C.byref(n), k, *[a.ctypes.data_as(_I) for a in arrs]),
              "lhmm_micro_plan")
        return [dict(boxes=int(arrs[0][c]), max_beads=int(arrs[1][c]), threads=int(arrs[2][c]),
                     min_blocks=int(arrs[3][c])) for c in range(k)]

    def set_variant(self, cls, variant):
        check(lib().lhmm_micro_set_variant(self.h, int(cls), int(variant)),
              "lhmm_micro_set_variant")

    def set_list_variant(self, variant=-1):
        """Kernel variant of the launches over a box list.  -1 restores the
        default: up to one listed box per SM, one block per SM with the most
        threads that fit; more boxes, two 512-thread blocks per SM."""
        check(lib().lhmm_micro_set_list_variant(self.h, int(variant)),
              "lhmm_micro_set_list_variant")

    def info(self):
        nb = C.c_int()
        tot = C.c_int64()
        mx = C.c_int()
        check(lib().lhmm_micro_info(self.h, C.byref(nb), C.byref(tot), C.byref(mx)),
              "lhmm_micro_info")
        return nb.value, tot.value, mx.value


def sph_params(n, n_wall=0, **kw):
    d = dict(Lx=1.0, Ly=1.0, h=0.3, mass=1.0, rho0=1.0, c=1.0, theta_pb=0.1, eta_s=0.1,
             zeta_s=0.0, dt=1e-3, kernel=SPH_WENDLAND_C2, visc_coeffs=SPH_VISC_DERIVED_2D,
             body_mode=SPH_BODY_UNIFORM)
    bf = kw.pop("body_force", (0.0, 0.0))
    d.update(kw)
    p = SphParams(n=int(n), n_wall=int(n_wall), **d)
    p.body_force[0], p.body_force[1] = bf
    return p


class Sph:
    """Macroscale SPH particles resident on the GPU (lhmm_sph_*)."""

    def __init__(self, params, pos0, vel0, stream=None):
        pos0, pp = _np(np.asarray(pos0, np.float32).reshape(-1, 2), np.float32)
        vel0, pv = _np(np.asarray(vel0, np.float32).reshape(-1, 2), np.float32)
        self.params = params
        self.n = int(params.n)
        self.n_fluid = int(params.n - params.n_wall)
        h = C.c_void_p()
        check(lib().lhmm_sph_create(C.byref(params), pp, pv, _stream_ptr(stream), C.byref(h)),
              "lhmm_sph_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().lhmm_sph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n_substeps, stress_dev=None, L_out_dev=None, stream=None):
        check(lib().lhmm_sph_step(self.h, _ptr(stress_dev), int(n_substeps), _ptr(L_out_dev),
                                  _stream_ptr(stream)), "lhmm_sph_step")

    def recompute_forces(self, stress_dev=None, stream=None):
        check(lib().lhmm_sph_recompute_forces(self.h, _ptr(stress_dev), _stream_ptr(stream)),
              "lhmm_sph_recompute_forces")

    def get_state(self):
        pos = np.zeros((self.n, 2), np.float32)
        vel = np.zeros((self.n, 2), np.float32)
        acc = np.zeros((self.n, 2), np.float32)
        d = np.zeros(self.n, np.float32)
        check(lib().lhmm_sph_get_state(self.h, pos.ctypes.data_as(_F), vel.ctypes.data_as(_F),
                                       acc.ctypes.data_as(_F), d.ctypes.data_as(_F)),
              "lhmm_sph_get_state")
        return pos, vel, acc, d




# micro kernel variants (include/lhmm.h): threads per block, resident blocks
# per SM, and whether the box arrays live in device memory instead of shared
MICRO_VARIANTS = [(256, 4, False), (512, 2, False), (1024, 1, False), (256, 2, False),
                  (512, 1, False), (512, 1, True), (256, 2, True)]

NOALLOC_MAX_PARTICLES = 65536


def sph_velgrad_noalloc(params, pos_dev, vel_dev, L_out_dev, stream=None):
    """Velocity gradients of the given particles without any device allocation
    (lhmm_sph_velgrad_noalloc): for callers that may not allocate device memory
    at that point.  All calls share one fixed scratch array in the library, so
    calls that may overlap on the GPU must be serialised by the caller."""
    check(lib().lhmm_sph_velgrad_noalloc(C.byref(params), _ptr(pos_dev), _ptr(vel_dev),
                                         _ptr(L_out_dev), _stream_ptr(stream)),
          "lhmm_sph_velgrad_noalloc")


class Coupled:
    """The LHMM macro step over an Sph and a Micro handle (lhmm_coupled_*)."""

    def __init__(self, sph, micro, sph_substeps, micro_steps):
        h = C.c_void_p()
        check(lib().lhmm_coupled_create(sph.h, micro.h, int(sph_substeps), int(micro_steps),
                                        C.byref(h)), "lhmm_coupled_create")
        self.h = h
        self.sph, self.micro = sph, micro  # keep the handles alive
        self.n_boxes = micro.n_boxes

    def close(self):
        if getattr(self, "h", None):
            lib().lhmm_coupled_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n_macro=1, use_graph=True, stream=None):
        check(lib().lhmm_coupled_step(self.h, int(n_macro), int(bool(use_graph)),
                                      _stream_ptr(stream)), "lhmm_coupled_step")

    def exchange_ptrs(self):
        Lp = C.c_void_p()
        sp = C.c_void_p()
        check(lib().lhmm_coupled_exchange(self.h, C.byref(Lp), C.byref(sp)),
              "lhmm_coupled_exchange")
        return Lp.value, sp.value

    def set_closure(self, closure, threshold=0.02, stress_floor=1e-3, audit_every=50):
        check(lib().lhmm_coupled_set_closure(self.h, closure.h, float(threshold),
                                             float(stress_floor), int(audit_every)),
              "lhmm_coupled_set_closure")
        self.closure = closure

    def set_online_calibration(self, enabled=True, decay=0.9):
        """Trusted boxes take a p + c, the line fitted to the audited boxes'
        DPD values on their raw predictions (enabled=-1 only reads the map).
        Returns the current (a, c) of xx, xy, yy as a 3 x 2 array."""
        m = np.zeros(6, np.float32)
        check(lib().lhmm_coupled_set_online_calibration(self.h, int(enabled), float(decay),
                                                        m.ctypes.data_as(_F)),
              "lhmm_coupled_set_online_calibration")
        return m.reshape(3, 2)

    def enable_gate(self, on=True):
        check(lib().lhmm_coupled_enable_gate(self.h, int(bool(on))), "lhmm_coupled_enable_gate")

    def set_gate(self, threshold, audit_every=50, absolute=False, warmup_steps=-1):
        check(lib().lhmm_coupled_set_gate(self.h, float(threshold), int(audit_every),
                                          int(bool(absolute)), int(warmup_steps)),
              "lhmm_coupled_set_gate")

    def gate_stats(self):
        a, b_, c_ = C.c_int64(), C.c_int64(), C.c_int64()
        e, r = C.c_double(), C.c_double()
        check(lib().lhmm_coupled_gate_stats(self.h, C.byref(a), C.byref(b_), C.byref(c_),
                                            C.byref(e), C.byref(r)), "lhmm_coupled_gate_stats")
        return dict(gated_steps=a.value, dpd_boxes=b_.value, audited=c_.value,
                    audit_err2=e.value, audit_ref2=r.value)

    def closure_inputs(self):
        X = np.zeros((self.n_boxes, 67), np.float32)
        check(lib().lhmm_coupled_closure_inputs(self.h, X.ctypes.data_as(_F)),
              "lhmm_coupled_closure_inputs")
        return X

    def exchange(self):
        """Host copies of the exchange buffers (waits for the device)."""
        L = np.zeros((self.n_boxes, 9), np.float32)
        st = np.zeros((self.n_boxes, 6), np.float64)
        check(lib().lhmm_coupled_copy_exchange(self.h, L.ctypes.data_as(_F),
                                               st.ctypes.data_as(_D)), "lhmm_coupled_copy_exchange")
        return L, st


class Closure:
    """Ensemble MLP stress closure trained and evaluated on the GPU (lhmm_closure_*)."""

    def __init__(self, members=5, in_dim=67, hidden=256, n_hidden=4, out_dim=3, seed=1):
        h = C.c_void_p()
        check(lib().lhmm_closure_create(members, in_dim, hidden, n_hidden, out_dim, seed,
                                        C.byref(h)), "lhmm_closure_create")
        self.h = h
        self.members, self.in_dim, self.out_dim = members, in_dim, out_dim
        self.dims = [in_dim] + [hidden] * n_hidden + [out_dim]
        n = C.c_int64()
        check(lib().lhmm_closure_info(h, C.byref(n), None), "lhmm_closure_info")
        self.n_params = n.value

    def close(self):
        if getattr(self, "h", None):
            lib().lhmm_closure_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_gemm(self, path):
        """1: tcgen05 tensor-core products (default); 0: mma.sync products."""
        check(lib().lhmm_closure_set_gemm(self.h, int(path)), "lhmm_closure_set_gemm")

    def sync(self):
        check(lib().lhmm_closure_sync(self.h), "lhmm_closure_sync")

    def set_normalization(self, in_mean, in_std, out_scale):
        a, pa = _np(in_mean, np.float32)
        b_, pb = _np(in_std, np.float32)
        c_, pc = _np(out_scale, np.float32)
        check(lib().lhmm_closure_set_normalization(self.h, pa, pb, pc),
              "lhmm_closure_set_normalization")

    def train_step(self, X_dev, T_dev, B, lr, weight_decay=0.0, rows_dev=None, loss_dev=None,
                   stream=None):
        check(lib().lhmm_closure_train_step(self.h, _ptr(X_dev), _ptr(T_dev), _ptr(rows_dev),
                                            int(B), float(lr), float(weight_decay),
                                            _ptr(loss_dev), _stream_ptr(stream)),
              "lhmm_closure_train_step")

    def infer(self, X_dev, mean_dev, spread_dev, stream=None):
        check(lib().lhmm_closure_infer(self.h, _ptr(X_dev), int(X_dev.shape[0]), _ptr(mean_dev),
                                       _ptr(spread_dev), _stream_ptr(stream)), "lhmm_closure_infer")

    def forward_members(self, X_dev):
        n = int(X_dev.shape[0])
        Y = np.zeros((self.members, n, self.out_dim), np.float32)
        check(lib().lhmm_closure_forward(self.h, _ptr(X_dev), n, Y.ctypes.data_as(_F)),
              "lhmm_closure_forward")
        return Y

    def get_params(self, member=0):
        p = np.zeros(self.n_params, np.float32)
        check(lib().lhmm_closure_get_params(self.h, int(member), p.ctypes.data_as(_F)),
              "lhmm_closure_get_params")
        return p

    def set_params(self, member, params):
        p, pp = _np(params, np.float32)
        check(lib().lhmm_closure_set_params(self.h, int(member), pp), "lhmm_closure_set_params")

    def get_grad(self, member=0):
        g = np.zeros(self.n_params, np.float32)
        check(lib().lhmm_closure_get_grad(self.h, int(member), g.ctypes.data_as(_F)),
              "lhmm_closure_get_grad")
        return g
