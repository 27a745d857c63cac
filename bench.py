"""Benchmark of the batched DPD micro step (the LHMM micro hot path).

One step = one lhmm_micro_advance call that advances every box of the
batched-microsolver workload (1024 AFBC boxes, edges uniform in {6..12},
about 2.57M beads, 20 % of them in N_d = 10 FENE chains, per-box velocity
gradients) by 100 DPD steps and returns per-box time-averaged IK stress.

Prints one JSON line (rank 0).  Under torchrun every rank runs its own
batch of the same shape (weak scaling, no data-path collective).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reference arm of this
build) on a bounded sample of the same workload on the host cores.

Beside the main metric, rank 0 adds these entries to the line.  Each
comes after the timed region, and a flag skips it:
  cpu_baseline   the oracle on a 10 s sample of the workload (--no-cpu-baseline)
  secondary, rpf_paper, rpm_paper
                 macro-steps/s of the coupled channel, of the paper's
                 reverse-Poiseuille set-up and of its porous-medium scale
                 (--no-macro)
  surrogate      plain vs surrogate-gated channel: closure trained on 2.05M
                 pairs for 20k steps, gate threshold 0.1 with online
                 calibration, profile errors and noise floor (about two
                 minutes; --no-surrogate)
  large_mixed    plain vs gated cylinder array with 16.4M beads, 200 macro
                 steps each (--no-large-mixed)

  python bench.py --profile-case micro|mlp|sph|gated

runs one fixed, small invocation of a kernel family for a profiler to
capture and exits 0 without a bench line: micro = 304 boxes of edge 12
(5184 beads) for 3 calls of 10 DPD steps; mlp = 4 closure training steps at
B = 4096 and one inference of 16 384 rows; sph = 3 x 20 substeps of a
cylinder cell with 16 384 fluid particles; gated = 3 surrogate-gated macro
steps of the coupled channel with 1 in 14 boxes on DPD.
"""
import ctypes
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DPD bead-steps/s (batched micro boxes)"
UNIT = "bead-steps/s"
MICRO_STEPS = 100
# Algorithmic operations per bead-step, counting only what the method must
# do (each unique interacting pair once, no rejected candidates): per pair
# ~40 FP32 operations (distance 8, rsqrt 1, w 2, conservative 2, dissipative
# 7, random scale 4, forces on i and j 6, virial 9), ~60 integer operations
# (Philox4x32-10, two of its four words used) and 3 SFU calls (log, sqrt,
# cos); per bead ~40 FP32 operations (FENE, two half kicks, drift, IK
# kinetic part).  At rho = 3 a bead has rho (4 pi / 3) rc^3 / 2 = 6.28 unique
# partners: 291 FP32 + 377 int + 19 SFU = 687 operations per bead-step.
PAIRS_PER_BEAD = 2.0 * np.pi / 3.0 * 3.0
FP32_PER_PAIR, INT_PER_PAIR, SFU_PER_PAIR, FP32_PER_BEAD = 40, 60, 3, 40
ALGO_OPS_PER_BEAD_STEP = PAIRS_PER_BEAD * (FP32_PER_PAIR + INT_PER_PAIR + SFU_PER_PAIR) + FP32_PER_BEAD
# The same work recounted per issued instruction of a plain implementation
# (Philox as separate multiply-high, multiply-low, xor and key-add
# instructions: 159 per pair, 35 per bead), reported beside it.
ISSUED_OPS_PER_BEAD_STEP = PAIRS_PER_BEAD * 159 + 35
LANES_PER_SM_CLK = 128  # FP32/INT32 lanes of an SM (4 sub-partitions x 32)
# DRAM bytes (read + write) per bead and call of micro_kernel, from the ncu
# capture in profiles/micro_kernel_e12_304box_full.md (75.84 + 16.04 MB for
# 1,575,936 beads); the kernel reads and writes box state once per call, so
# traffic scales with beads, not with DPD steps.
DRAM_BYTES_PER_BEAD_CALL = 91.884e6 / 1575936


def build_probe(force=False):
    """Compile bench_probe.cu (the issue-rate probe of the roofline, a
    measurement helper outside the library) into bench_probe.so beside this
    file; returns its path."""
    src = os.path.join(ROOT, "bench_probe.cu")
    out = os.path.join(ROOT, "bench_probe.so")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    from paper_2512_13267_gb300 import build_ext
    tmp = out + ".tmp%d" % os.getpid()
    cmd = [build_ext._nvcc()] + build_ext.ARCH + ["-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                                                   "-shared", src, "-o", tmp, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for bench_probe.cu:\n" + r.stdout + r.stderr)
    os.replace(tmp, out)
    return out


def issue_rate_probe(stream_ptr, iters=200):
    """(FP32 FMA, int xor + add) lane-operations per second of this GPU."""
    lib = ctypes.CDLL(build_probe())
    f = lib.bench_issue_rate_probe
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                  ctypes.c_void_p]
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = f(int(iters), ctypes.byref(a), ctypes.byref(b), ctypes.c_void_p(stream_ptr))
    if rc != 0:
        raise RuntimeError("bench_issue_rate_probe failed: %d" % rc)
    return a.value, b.value


def profile_case_micro(boxes=304, edge=12.0, steps=10, calls=3):
    import torch
    from paper_2512_13267_gb300 import lhmm, synth
    batch = synth.make_batch(np.full(boxes, edge),
                             synth.random_velocity_gradients(boxes, seed=2), 2, flow="afbc")
    m = lhmm.Micro.from_batch(lhmm.dpd_params(flow="afbc", seed=2), batch)
    L = torch.from_numpy(batch.L).cuda()
    st = torch.zeros((boxes, 6), dtype=torch.float64, device="cuda")
    for _ in range(calls):
        m.advance(L, steps, st)
    torch.cuda.synchronize()
    m.close()


def profile_case_mlp(rows=4096, steps=4):
    import torch
    from paper_2512_13267_gb300 import lhmm
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


def profile_case_sph(n_fluid=16384, cell=16.0, substeps=20):
    import torch
    from paper_2512_13267_gb300 import lhmm, synth
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


def profile_case_gated(audit_every=14, steps=3):
    """Gated macro steps of the coupled channel (2048 particles, 1500-bead
    boxes): every box trusted by a closure whose increments are negligible,
    so the flow is the plain one and the DPD share is the audit share
    (1/audit_every); plain warm-up steps for the gradient history, then
    `steps` gated steps launched eagerly."""
    import torch
    from paper_2512_13267_gb300 import closure as CL
    kw = dict(alpha=0.01, U_o=0.25, c_factor=10.0, eta_s=0.1, k_micro=50, dt_dpd=0.01, members=5)
    cpl, clo, _, _ = CL._channel(seed=3, closure_seed=7, **kw)
    clo.set_normalization(np.zeros(CL.N_IN), np.ones(CL.N_IN), np.full(CL.N_OUT, 1e-9))
    cpl.set_closure(clo, threshold=1e30, audit_every=audit_every)
    cpl.step(17, use_graph=False)
    cpl.enable_gate(True)
    cpl.step(steps, use_graph=False)
    torch.cuda.synchronize()
    for o in (cpl, cpl.micro, cpl.sph, clo):
        o.close()


PROFILE_CASES = {"micro": profile_case_micro, "mlp": profile_case_mlp, "sph": profile_case_sph,
                 "gated": profile_case_gated}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def workload_desc(batch):
    return {"workload": "batched micro step: %d AFBC DPD/FENE boxes, edge U{6..12} r_c, "
                        "%d beads (rho 3, 20%% in N_d=10 chains), %d DPD steps per call"
                        % (batch.n_boxes, batch.total_beads, MICRO_STEPS),
            "boxes": batch.n_boxes, "beads": batch.total_beads, "micro_steps_per_step": MICRO_STEPS,
            "l2": "flushed (256 MiB write) between timed steps"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, n in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(batch, budget_s=20.0, min_s=10.0, chunk_steps=5, n_boxes=24):
    """FP64 oracle (OpenMP over boxes) on a fixed sample of the same workload.
    Returns (bead-steps/s, threads, description)."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O
    rng = np.random.default_rng(1234)
    ids = np.sort(rng.choice(batch.n_boxes, size=min(n_boxes, batch.n_boxes), replace=False))
    par = O.dpd_params(flow_mode=O.FLOW_AFBC, seed=2)
    boxes = []
    for b in ids:
        sl = batch.box_slice(int(b))
        ob = O.Box(batch.edges[b], batch.pos[sl], batch.vel[sl], int(batch.n_chains[b]),
                   batch.chain_len, box_id=int(b))
        O.compute_forces(par, ob, batch.L[b])
        boxes.append(ob)
    L = batch.L[ids].astype(np.float64)
    beads = int(sum(b.n for b in boxes))
    threads = O.max_threads()
    done = 0
    t0 = time.perf_counter()
    while True:
        O.advance_batch(par, boxes, L, chunk_steps, n_threads=threads)
        done += chunk_steps
        el = time.perf_counter() - t0
        if el >= min_s or el >= budget_s:
            break
    rate = beads * done / el
    desc = "%d of %d boxes (%d beads), %d DPD steps, %.1f s" % (len(ids), batch.n_boxes, beads,
                                                                 done, el)
    return rate, threads, desc


def cpu_oracle_macro_rate(sph_cfg, batch, eta_s, alpha, k_micro, n_sample=32):
    """FP64 oracles on the same coupled channel: one macro step of the SPH
    oracle over every particle (M substeps, density, velocity gradient) and
    k' DPD steps of the micro oracle (OpenMP over boxes) on a fixed sample of
    boxes, scaled to all boxes.  Returns (macro-steps/s, threads, description)."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O
    M = sph_cfg["substeps"]
    op = O.sph_params(n=sph_cfg["pos"].shape[0], Lx=sph_cfg["Lx"], Ly=sph_cfg["Ly"],
                      h=sph_cfg["h"], mass=sph_cfg["mass"], rho0=1.0, c=sph_cfg["c"],
                      theta_pb=0.1, eta_s=eta_s, zeta_s=0.0, dt=sph_cfg["dt"],
                      kernel=O.KERNEL_WENDLAND_C2,
                      visc_coeffs=O.VISC_DERIVED_2D, body_force=(sph_cfg["body_force"], 0.0),
                      body_mode=O.BODY_REVERSE_POISEUILLE)
    pos = sph_cfg["pos"].astype(np.float64)
    vel = sph_cfg["vel"].astype(np.float64)
    t0 = time.perf_counter()
    acc, _ = O.sph_accel(op, pos, vel)
    O.sph_steps(op, pos, vel, acc, M)
    d = O.sph_density(op, pos)
    O.sph_velgrad(op, pos, vel, d)
    t_sph = time.perf_counter() - t0
    par = O.dpd_params(flow_mode=O.FLOW_AFBC, seed=3, alpha=alpha)
    ids = np.arange(min(n_sample, batch.n_boxes))
    boxes = []
    for b in ids:
        sl = batch.box_slice(int(b))
        ob = O.Box(batch.edges[b], batch.pos[sl], batch.vel[sl], int(batch.n_chains[b]),
                   batch.chain_len, box_id=int(b))
        O.compute_forces(par, ob, np.zeros(9))
        boxes.append(ob)
    threads = O.max_threads()
    t0 = time.perf_counter()
    O.advance_batch(par, boxes, np.zeros((len(ids), 9)), k_micro, n_threads=threads)
    t_micro = (time.perf_counter() - t0) * batch.n_boxes / len(ids)
    desc = ("SPH oracle: one macro step of all %d particles (%d substeps, %.1f s); micro "
            "oracle: %d of %d boxes for %d DPD steps, scaled to all boxes (%.1f s)"
            % (pos.shape[0], M, t_sph, len(ids), batch.n_boxes, k_micro, t_micro))
    return 1.0 / (t_sph + t_micro), threads, desc


def macro_step_rate(steps=10, warmup=2, cpu_oracle=False):
    """LHMM macro-steps/s of the coupled reverse-Poiseuille channel (64 x 32 SPH
    particles, one 1500-bead AFBC box each, k' = 50 DPD steps per macro step,
    M SPH substeps from the CFL rule), graph-captured macro steps."""
    import torch
    from paper_2512_13267_gb300 import lhmm, synth
    U_o, c_fac, eta_s, alpha, k_micro, dt_dpd = 0.25, 10.0, 0.1, 0.01, 50, 0.01
    sph_cfg, batch = synth.coupled_channel(U_o=U_o, c_factor=c_fac, eta_s=eta_s,
                                           delta_t=k_micro * dt_dpd)
    M = sph_cfg["substeps"]
    sp = lhmm.sph_params(sph_cfg["pos"].shape[0], 0, Lx=sph_cfg["Lx"], Ly=sph_cfg["Ly"],
                         h=sph_cfg["h"], mass=sph_cfg["mass"], rho0=1.0, c=sph_cfg["c"],
                         theta_pb=0.1, eta_s=eta_s, dt=sph_cfg["dt"],
                         body_force=(sph_cfg["body_force"], 0.0),
                         body_mode=lhmm.SPH_BODY_REVERSE_POISEUILLE)
    sph = lhmm.Sph(sp, sph_cfg["pos"], sph_cfg["vel"])
    micro = lhmm.Micro.from_batch(lhmm.dpd_params(flow="afbc", seed=3, alpha=alpha), batch)
    L0 = torch.zeros((batch.n_boxes, 9), dtype=torch.float32, device="cuda")
    micro.autotune(L0, probe_steps=10)
    cpl = lhmm.Coupled(sph, micro, M, k_micro)
    stream = torch.cuda.current_stream()
    cpl.step(warmup, use_graph=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cpl.step(steps, use_graph=True)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    status, _ = micro.sync(raise_on_error=False)
    out = {"metric": "LHMM macro-steps/s (plain DPD closure)", "value": steps / (ms / 1e3),
           "unit": "macro-steps/s", "ms_per_macro_step": ms / steps, "steps": steps,
           "warmup": warmup, "sph_particles": int(sph_cfg["pos"].shape[0]),
           "sph_substeps": M, "micro_steps": k_micro, "boxes": batch.n_boxes,
           "beads": batch.total_beads,
           "bead_steps_per_s": batch.total_beads * k_micro * steps / (ms / 1e3),
           "cuda_graph": True, "device_status": lhmm.status_string(status),
           "workload": "coupled reverse-Poiseuille channel 64x32 SPH (Ly=4, h=3dh, Wendland, "
                       "c=10 U_o, U_o=0.25, eta_s=0.1) x 1500-bead AFBC boxes, k'=50, M=%d" % M}
    cpl.close()
    micro.close()
    sph.close()
    if cpu_oracle:
        rate, threads, desc = cpu_oracle_macro_rate(sph_cfg, batch, eta_s, alpha, k_micro)
        out["cpu_baseline"] = {"value": rate, "unit": "macro-steps/s", "cores": threads,
                               "kind": "oracle", "sample": desc}
    return out


def sharded_macro_rate(world, rank, steps=10, warmup=2):
    """LHMM macro-steps/s of one coupled reverse-Poiseuille channel (the
    `secondary` workload) spread over the ranks: SPH replicated, the 2048
    boxes in bead-balanced ranges, one NCCL all-gather of the n x 6 stresses
    per macro step (strong scaling of one system)."""
    import torch
    import torch.distributed as dist
    from paper_2512_13267_gb300 import lhmm, sharding, synth
    U_o, c_fac, eta_s, alpha, k_micro, dt_dpd = 0.25, 10.0, 0.1, 0.01, 50, 0.01
    cfg, batch = synth.coupled_channel(U_o=U_o, c_factor=c_fac, eta_s=eta_s,
                                       delta_t=k_micro * dt_dpd)
    n, M = cfg["pos"].shape[0], cfg["substeps"]
    sp = lhmm.sph_params(n, 0, Lx=cfg["Lx"], Ly=cfg["Ly"], h=cfg["h"], mass=cfg["mass"],
                         rho0=1.0, c=cfg["c"], theta_pb=0.1, eta_s=eta_s, dt=cfg["dt"],
                         body_force=(cfg["body_force"], 0.0),
                         body_mode=lhmm.SPH_BODY_REVERSE_POISEUILLE)
    sph = lhmm.Sph(sp, cfg["pos"], cfg["vel"])
    ranges = sharding.partition_boxes(batch.n_beads, world)
    lo, hi = ranges[rank]
    micro = lhmm.Micro.from_batch(lhmm.dpd_params(flow="afbc", seed=3, alpha=alpha),
                                  batch.boxes(lo, hi), box_id_offset=lo)
    drv = sharding.ShardedCoupled(sharding.GpuSph(sph, n, M), sharding.GpuMicro(micro, k_micro),
                                  ranges, torch.zeros((n, 6), dtype=torch.float64, device="cuda"))
    drv.step(warmup)
    torch.cuda.synchronize()
    dist.barrier()
    t0 = time.perf_counter()
    drv.step(steps)
    torch.cuda.synchronize()
    dist.barrier()
    t = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    micro.close()
    sph.close()
    return {"metric": "LHMM macro-steps/s, one coupled channel sharded over the ranks",
            "value": steps / float(t.item()), "unit": "macro-steps/s", "ranks": world,
            "boxes_per_rank": [b - a for a, b in ranges], "scaling": "strong",
            "workload": "coupled reverse-Poiseuille channel 64x32 SPH x 1500-bead AFBC boxes, "
                        "k'=50, M=%d; SPH replicated, boxes sharded, stress all-gather" % M}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2512_13267_gb300 import synth
    batch = synth.batched_microsolver()
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O
    rng = np.random.default_rng(1234)
    ids = np.sort(rng.choice(batch.n_boxes, size=16, replace=False))
    par = O.dpd_params(flow_mode=O.FLOW_AFBC, seed=2)
    boxes = []
    for b in ids:
        sl = batch.box_slice(int(b))
        ob = O.Box(batch.edges[b], batch.pos[sl], batch.vel[sl], int(batch.n_chains[b]),
                   batch.chain_len, box_id=int(b))
        O.compute_forces(par, ob, batch.L[b])
        boxes.append(ob)
    L = batch.L[ids].astype(np.float64)
    beads = int(sum(b.n for b in boxes))
    threads = O.max_threads()
    steps_per = 10
    for _ in range(args.warmup):
        O.advance_batch(par, boxes, L, steps_per, n_threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.advance_batch(par, boxes, L, steps_per, n_threads=threads)
    el = time.perf_counter() - t0
    value = beads * steps_per * args.steps / el
    cfg = workload_desc(batch)
    sample = ("each step: %d sampled boxes (%d beads) x %d DPD steps of the %d-box workload"
              % (len(ids), beads, steps_per, batch.n_boxes))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--boxes", type=int, default=1024,
                    help="boxes of the workload (a smaller case for profilers)")
    ap.add_argument("--micro-steps", type=int, default=100, help="DPD steps per call")
    ap.add_argument("--no-macro", action="store_true", help="skip the coupled macro-step line")
    ap.add_argument("--no-surrogate", action="store_true",
                    help="skip the surrogate-gated vs plain comparison")
    ap.add_argument("--no-large-mixed", action="store_true",
                    help="skip the large mixed run (cylinder array, 16.4 M beads, gated)")
    ap.add_argument("--uniform-edge", type=float, default=0.0,
                    help="give every box this edge (a one-class case for profilers)")
    ap.add_argument("--profile-case", choices=sorted(PROFILE_CASES),
                    help="run one fixed small invocation for a profiler and exit")
    args = ap.parse_args()
    if args.profile_case:
        PROFILE_CASES[args.profile_case]()
        return 0
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_2512_13267_gb300 import lhmm, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    lhmm.lib()

    global MICRO_STEPS
    MICRO_STEPS = args.micro_steps
    if args.uniform_edge > 0:
        batch = synth.make_batch(np.full(args.boxes, args.uniform_edge),
                                 synth.random_velocity_gradients(args.boxes, 2 + rank), 2 + rank)
    else:
        batch = synth.batched_microsolver(n_boxes=args.boxes, seed=2 + rank)
    params = lhmm.dpd_params(flow="afbc", seed=2 + rank)
    micro = lhmm.Micro.from_batch(params, batch)
    stream = torch.cuda.current_stream()
    L = torch.from_numpy(batch.L).cuda()
    stress = torch.zeros((batch.n_boxes, 6), dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2

    micro.autotune(L, probe_steps=10)  # launch plan: size classes or one persistent launch (state restored)
    for _ in range(max(args.warmup, 0)):
        micro.advance(L, MICRO_STEPS, stress)
    torch.cuda.synchronize()
    # over-stretch under strong extension is reported below
    _, warm_status = micro.sync(raise_on_error=False)

    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    evs = []
    for k in range(args.steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        micro.advance(L, MICRO_STEPS, stress)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    times_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = float(sum(times_ms))
    status, timed_status = micro.sync(raise_on_error=False)
    clamped = int(np.count_nonzero((warm_status | timed_status) & lhmm.BOX_BOND_OVERSTRETCH))
    t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    bead_steps_rank = batch.total_beads * MICRO_STEPS * args.steps
    # every rank's batch has its own seed, so the bead counts differ a little:
    # the job's value is all ranks' bead-steps over the slowest rank's time
    bs = torch.tensor([float(bead_steps_rank)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(bs, op=dist.ReduceOp.SUM)
    value = float(bs.item()) / (max_ms / 1e3)

    # end to end through the host-buffer entry point (pinned buffers)
    L_pin = torch.from_numpy(batch.L).pin_memory()
    st_pin = torch.zeros((batch.n_boxes, 6), dtype=torch.float64).pin_memory()
    micro.advance_host(L_pin.numpy(), MICRO_STEPS, st_pin.numpy())
    e2e_steps = max(2, min(args.steps, 3))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        micro.advance_host(L_pin.numpy(), MICRO_STEPS, st_pin.numpy())
    e2e_s = time.perf_counter() - t0
    e2e = torch.tensor([e2e_s, float(batch.total_beads * MICRO_STEPS * e2e_steps)],
                       dtype=torch.float64, device="cuda")
    if world > 1:  # slowest rank's wall time, all ranks' bead-steps
        t_max = e2e[:1].clone()
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
        dist.all_reduce(e2e, op=dist.ReduceOp.SUM)
        e2e[0] = t_max[0]
    e2e_val = float(e2e[1].item()) / float(e2e[0].item())

    peaks, src = _peaks()
    clk_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = n_sm * LANES_PER_SM_CLK * clk_mhz * 1e6 / 1e12  # T lane-ops/s
    per_launch_ops = ALGO_OPS_PER_BEAD_STEP * batch.total_beads * MICRO_STEPS
    launch_s = (total_ms / args.steps) / 1e3
    achieved = per_launch_ops / launch_s / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                "frac": achieved / alu_peak,
                "traffic": DRAM_BYTES_PER_BEAD_CALL * batch.total_beads,
                "traffic_unit": "bytes per call (every micro_kernel launch of the call), scaled "
                                "by beads from the 304-box capture",
                "peak_source": "%d SMs (queried) x %d FP32/INT lanes x %.0f MHz (%s sm_max_mhz)"
                               % (n_sm, LANES_PER_SM_CLK, clk_mhz, src),
                "kernel": "micro_kernel", "algo_ops_per_bead_step": ALGO_OPS_PER_BEAD_STEP,
                "algo_ops_split": "%.0f FP32 + %.0f int + %.0f SFU per bead-step"
                                  % (PAIRS_PER_BEAD * FP32_PER_PAIR + FP32_PER_BEAD,
                                     PAIRS_PER_BEAD * INT_PER_PAIR, PAIRS_PER_BEAD * SFU_PER_PAIR),
                "frac_issued_recount": (ISSUED_OPS_PER_BEAD_STEP / ALGO_OPS_PER_BEAD_STEP)
                                       * achieved / alu_peak,
                "issued_ops_per_bead_step": ISSUED_OPS_PER_BEAD_STEP}
    try:  # measured issue rate of the CUDA cores, beside the derived peak
        f_rate, i_rate = issue_rate_probe(stream.cuda_stream, iters=200)
        roofline["probe_ffma_tops"] = f_rate / 1e12
        roofline["probe_int_xor_add_tops"] = i_rate / 1e12
        roofline["frac_of_int_probe"] = achieved / (i_rate / 1e12)
    except Exception as exc:  # pragma: no cover
        roofline["probe_error"] = str(exc)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_desc(batch), "roofline": roofline,
            "e2e": {"value": e2e_val, "unit": UNIT,
                    "h2d_bytes_per_step": int(L_pin.numel() * 4),
                    "d2h_bytes_per_step": int(st_pin.numel() * 8)},
            "gpu_launches": args.steps * len(micro.plan()),
            "launch_plan": micro.plan(), "device_status": lhmm.status_string(status),
            "bond_clamped_boxes": clamped,
            "bond_clamp_note": ("%d of %d boxes (planar extension at the highest rates) had a FENE "
                                "bond reach R0 in the warm-up or timed calls; their bond stiffness "
                                "is held at the (r/R0)^2 = 0.99 value (reading R10), the oracle "
                                "flags the same boxes" % (clamped, batch.n_boxes))}
    if clk is not None:
        line["clocks"] = clk
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, desc = cpu_oracle_rate(batch)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": desc}
    micro.close()
    if world > 1 and not args.no_macro and args.uniform_edge <= 0:
        line["coupled_sharded"] = sharded_macro_rate(world, rank)
    if rank == 0 and not args.no_macro and args.uniform_edge <= 0:
        line["secondary"] = macro_step_rate(cpu_oracle=not args.no_cpu_baseline)
        from paper_2512_13267_gb300 import flows
        line["rpf_paper"] = flows.rpf_paper_rate()
        # the paper's largest run (random porous medium, 76 x 76 boxes of
        # N_d = 16 melt): its 65.7 h for ~1.41e5 SPH steps is 1.68 s per SPH
        # step, 84 s per macro step of M = 50 substeps, for 12 288 boxes
        rpm = flows.rpm_paper_rate(steps=3, warmup=1)
        rpm["paper_s_per_macro_step"] = 1.68 * 50
        rpm["paper_beads"] = 12288 * 23104
        rpm["paper_bead_steps_per_s"] = 12288 * 23104 * 25 / (1.68 * 50)
        line["rpm_paper"] = rpm
    if rank == 0 and not args.no_surrogate and args.uniform_edge <= 0:
        from paper_2512_13267_gb300 import closure
        r = closure.surrogate_vs_plain(warm=20, n_data=1000, train_steps=20000, n_eval=60,
                                       absolute=True, calibrated=True, weight_decay=0.0,
                                       threshold=0.1, online_calibration=True, noise_floor=True)
        for k in ("profile_pxy_plain", "profile_pxy_surrogate"):
            r.pop(k, None)
        r["metric"] = "LHMM macro-steps/s, surrogate-gated vs plain"
        r["budget"] = ("1000 macro steps of training pairs (2.05M pairs), 20000 AdamW steps, "
                       "stress target, held-out calibration, gate threshold 0.1 with online "
                       "calibration from the audits (2% round-robin), warm-up k' steps for "
                       "boxes that return to DPD")
        line["surrogate"] = r
    if rank == 0 and not args.no_large_mixed and args.uniform_edge <= 0:
        # the large mixed run: periodic cylinder array, 16 384 fluid + wall
        # particles, 1000-bead boxes (16.4 M beads), graph-captured macro
        # steps, autotuned launch plan, 200 plain and 200 gated macro steps
        from paper_2512_13267_gb300 import closure
        r = closure.large_mixed_run(timing_steps=200, seed=5)
        r["metric"] = "LHMM macro-steps/s, large mixed run, surrogate-gated vs plain"
        line["large_mixed"] = r
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
