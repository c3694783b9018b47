"""Benchmark of the fused GI-filtered lattice Boltzmann step on one or more GB300s.

Default workload: D3Q19 periodic 256^3, FP32 storage and arithmetic, Taylor-Green
vortex u0 = 0.05, tau = 0.55, truncation order K = 2.  A "step" is one fused
pull-stream + collision pass over the whole lattice.  The metric is MLUPS
(million lattice-cell updates per second, whole job); the roofline is the HBM
bandwidth (2 Q sizeof(storage) algorithmic bytes per cell update).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead, on the host cores, on a bounded sample of the same workload.
Multi-GPU runs are independent replicas (one lattice per rank; the method has no
exchange between independent solves), launched with torchrun.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

LATTICE_Q = {"D2Q9": 9, "D3Q15": 15, "D3Q19": 19, "D3Q27": 27, "D3Q39": 39}
LATTICE_T0 = {"D2Q9": 1.0 / 3.0, "D3Q15": 1.0 / 3.0, "D3Q19": 1.0 / 3.0, "D3Q27": 1.0 / 3.0, "D3Q39": 2.0 / 3.0}
STORE_BYTES = {"f32": 4, "f16": 2, "bf16": 2, "f64": 8, "q16": 2}
DTYPE_NAME = {"f32": "f32", "f16": "f32 (f16 storage)", "bf16": "f32 (bf16 storage)", "f64": "f64",
              "q16": "f32 (16-bit fixed-point storage)"}
NOMINAL_HBM_GBS = 8000.0  # GB300 HBM3e, nominal (the measured copy peak is the roofline's denominator)
Q16_RANGE = 0.25  # fixed-point range for the Taylor-Green workloads (u0 = 0.05: |h| up to about 0.16)
KERNEL_SOURCES = ["lbm_core.cuh", "lbm_kernels.cuh", "lbm_lattice.cuh"]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--lattice", default="D3Q19", choices=list(LATTICE_Q))
    p.add_argument("--dims", type=int, nargs=3, default=[256, 256, 256])
    p.add_argument("--K", type=int, default=2)
    p.add_argument("--tau", type=float, default=0.55)
    p.add_argument("--u0", type=float, default=0.05)
    p.add_argument("--storage", default="f32", choices=list(STORE_BYTES))
    p.add_argument("--storage-range", type=float, default=Q16_RANGE, help="range of the q16 storage (power of two)")
    p.add_argument("--variant", type=int, default=None, help="force a kernel variant (default: autotune)")
    p.add_argument("--cpt", type=int, default=None, help="force cells per thread (with --variant 0)")
    p.add_argument("--block", type=int, default=None)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU work of the oracle sample")
    p.add_argument("--no-extras", action="store_true", help="skip the per-lattice and serving measurements")
    p.add_argument("--serve", type=int, default=200,
                   help="requests of the serving trace (2000 = the full Poisson workload; 0 = skip)")
    p.add_argument("--serve-rate", type=float, default=50.0)
    p.add_argument("--extra-steps", type=int, default=200)
    p.add_argument("--precision-report", action="store_true",
                   help="error of every storage form against FP64 storage on the headline, Galilean-invariance "
                        "and 512^3 workloads")
    return p.parse_args()


# (label, lattice, dims, K, tau, fields, steps, fixed-point range): the precision report's workloads.
# fields: ("tg", u0) = Taylor-Green; ("shear", U) = u_y = 0.01 sin(2 pi x / n) on a background U_x.
PRECISION_CONFIGS = [
    ("D3Q19 256^3 Taylor-Green u0=0.05 tau=0.55 K=2, 1000 steps", "D3Q19", (256, 256, 256), 2, 0.55,
     ("tg", 0.05), 1000, 0.25),
    ("D3Q27 192^3 shear wave 0.01 on U_x=0.1, tau=0.6 K=3, 2000 steps", "D3Q27", (192, 192, 192), 3, 0.6,
     ("shear", 0.1), 2000, 0.5),
    ("D3Q39 192^3 shear wave 0.01 on U_x=0.1, tau=0.6 K=4, 2000 steps", "D3Q39", (192, 192, 192), 4, 0.6,
     ("shear", 0.1), 2000, 1.0),
    ("D3Q19 512^3 Taylor-Green u0=0.05 tau=0.52 K=2, 500 steps", "D3Q19", (512, 512, 512), 2, 0.52,
     ("tg", 0.05), 500, 0.25),
]


def precision_report(stream):
    """Errors of the FP32, FP16, BF16 and 16-bit fixed-point storage forms (on the shear waves also
    fixed point shifted by the equilibrium at the background velocity) on each workload of
    PRECISION_CONFIGS, against the same run with FP64 storage and arithmetic (the FP64 oracle is
    too slow for these sizes; the library's FP64 path matches it within 1e-12 on the parity
    cases).  Taylor-Green: max|du| / max|u| and max|drho| / rho.  Shear wave: the same for the
    decaying component u_y, and the relative error of its Fourier amplitude at k = 1 (the
    quantity the decay-rate fit uses)."""
    import torch

    from paper_2002_02503_gb300 import fields, lbm

    report = []
    for label, lat, dims, K, tau, (kind, amp), steps, q_range in PRECISION_CONFIGS:
        if kind == "tg":
            rho, u = fields.taylor_green_3d(dims, amp, LATTICE_T0[lat])
        else:
            rho, u = fields.shear_wave(dims, 0.01, 3, 1, 0, background=(amp, 0.0, 0.0))
        out, ref = {}, None
        forms = ["f64", "f32", "f16", "bf16", "q16"]
        if kind == "shear":
            forms.append("q16_ref")  # automatic range, values stored relative to f^eq at U
        for storage in forms:
            shifted = storage == "q16_ref"
            s = lbm.Solver(lat, dims, tau, K, "q16" if shifted else storage, stream=stream,
                           storage_range=0.0 if shifted else (q_range if storage == "q16" else None),
                           storage_reference=(amp, 0.0, 0.0) if shifted else None)
            s.set_fields(rho, u)
            chosen = lbm.lbm_get_storage_range(s.handle) if storage.startswith("q16") else None
            s.step(steps)
            r, uu = s.moments()
            mode = s.mode((1, 0, 0), 1) if kind == "shear" else None
            s.close()
            del s
            torch.cuda.empty_cache()
            if kind == "shear":
                uu = uu[1]
            if ref is None:
                ref = (r, uu, mode)
                continue
            e = {"rel_u": float(np.max(np.abs(uu - ref[1])) / np.max(np.abs(ref[1]))),
                 "rel_rho": float(np.max(np.abs(r - ref[0]) / ref[0]))}
            if kind == "shear":
                e["rel_mode_amplitude"] = float(abs(abs(mode) - abs(ref[2])) / abs(ref[2]))
            if chosen is not None:
                e["range"] = chosen
            if shifted:
                e["reference"] = [amp, 0.0, 0.0]
            out[storage] = e
            del r, uu
        report.append({"workload": label, "errors": out})
        del rho, u
    return {"reference": "FP64 storage and arithmetic (same library)", "configs": report}


# (lattice, dims, K, storage, tau, u0): the other lattices and storages of the workload family
PER_LATTICE = [
    ("D3Q19", (256, 256, 256), 3, "f32", 0.55, 0.05),
    ("D3Q27", (192, 192, 192), 3, "f32", 0.6, 0.05),
    ("D3Q39", (192, 192, 192), 4, "f32", 0.6, 0.05),
    ("D3Q19", (512, 512, 512), 2, "f32", 0.52, 0.05),
    ("D3Q19", (512, 512, 512), 2, "f16", 0.52, 0.05),
    ("D3Q19", (512, 512, 512), 2, "bf16", 0.52, 0.05),
    ("D3Q19", (512, 512, 512), 2, "q16", 0.52, 0.05),
]

# The extensions of the method (energy-flux term, K = 5, D3Q15, the BGK comparison operator):
# (lattice, dims, K, storage, tau, u0, model, theta)
PER_MODE = [
    ("D3Q19", (256, 256, 256), 3, "f32", 0.6, 0.05, "filtered", 0.5),
    ("D3Q39", (192, 192, 192), 4, "f32", 0.6, 0.05, "filtered", 0.5),
    ("D3Q39", (192, 192, 192), 5, "f32", 0.6, 0.05, "filtered", 0.0),
    ("D3Q15", (256, 256, 256), 3, "f32", 0.6, 0.05, "filtered", 0.0),
    ("D3Q19", (256, 256, 256), 3, "f32", 0.6, 0.05, "bgk", 0.0),
    # fixed point on the shear waves of the Galilean-invariance workloads (0.01 on U_x = 0.1),
    # automatic range, without and with the reference shift at the background velocity
    ("D3Q27", (192, 192, 192), 3, "q16", 0.6, 0.1, "filtered", 0.0, "shear"),
    ("D3Q27", (192, 192, 192), 3, "q16", 0.6, 0.1, "filtered", 0.0, "shear_ref"),
    ("D3Q39", (192, 192, 192), 4, "q16", 0.6, 0.1, "filtered", 0.0, "shear"),
    ("D3Q39", (192, 192, 192), 4, "q16", 0.6, 0.1, "filtered", 0.0, "shear_ref"),
]


def measure_lattice(lattice, dims, K, storage, tau, u0, steps, stream, model="filtered", theta=0.0, field=None):
    """Autotuned MLUPS and HBM fraction of one configuration (CUDA events on the solver stream).
    model / theta: the collision operator (BGK comparison, energy-flux weight).  field: None for
    a Taylor-Green vortex of amplitude u0; "shear" for a 0.01 shear wave on the background
    U_x = u0 with the automatic fixed-point range; "shear_ref" the same with the fixed-point
    values stored relative to the equilibrium at the background."""
    import torch

    from paper_2002_02503_gb300 import fields, lbm

    if field is None:
        rho, u = fields.taylor_green_3d(dims, u0, LATTICE_T0[lattice])
        q_range, ref = Q16_RANGE, None
    else:
        rho, u = fields.shear_wave(dims, 0.01, 3, 1, 0, background=(u0, 0.0, 0.0))
        q_range, ref = 0.0, ((u0, 0.0, 0.0) if field == "shear_ref" else None)
    s = lbm.Solver(lattice, dims, tau, K, storage, stream=stream,
                   storage_range=q_range if storage == "q16" else None, storage_reference=ref)
    lbm.lbm_set_collision(s.handle, model)
    lbm.lbm_set_energy_flux(s.handle, theta)
    s.set_fields(rho, u)
    del rho, u
    lbm.lbm_autotune(s.handle, 10)
    variant, cpt, block = lbm.lbm_get_kernel(s.handle)
    s.step(5)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    s.close()
    del s
    torch.cuda.empty_cache()
    C = int(np.prod(dims))
    bpu = 2 * LATTICE_Q[lattice] * STORE_BYTES[storage]
    peak, _ = measured_peak()
    mlups = C * steps / (ms / 1e3) / 1e6
    mode = "" if model == "filtered" and theta == 0.0 else (" BGK" if model == "bgk" else " theta=%g" % theta)
    if field is not None:
        mode += " shear wave on U_x=%g%s" % (u0, ", reference shift" if field == "shear_ref" else "")
    return {"workload": "%s %dx%dx%d %s K=%d%s" % (lattice, dims[0], dims[1], dims[2], storage, K, mode),
            "MLUPS": mlups, "bytes_per_update": bpu, "achieved_GBs": mlups * 1e6 * bpu / 1e9,
            "frac_of_measured_hbm": mlups * 1e6 * bpu / 1e9 / peak, "ms_per_step": ms / steps,
            "kernel": {"variant": variant, "cells_per_thread": cpt, "block": block}}


def workload_name(a):
    return "%s periodic %dx%dx%d %s Taylor-Green u0=%g tau=%g K=%d" % (
        a.lattice, a.dims[0], a.dims[1], a.dims[2], a.storage.upper(), a.u0, a.tau, a.K)


def config_of(a, extra=None):
    c = {"workload": workload_name(a), "lattice": a.lattice, "dims": list(a.dims), "K": a.K, "tau": a.tau,
         "u0": a.u0, "storage": a.storage, "parallelism": "replicas",
         "l2": "inputs larger than L2: %.2f GB of distributions per step" % (
             2 * LATTICE_Q[a.lattice] * STORE_BYTES[a.storage] * int(np.prod(a.dims)) / 1e9)}
    if a.storage == "q16":
        c["storage_range"] = a.storage_range
    if extra:
        c.update(extra)
    return c


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def initial_fields(a):
    from paper_2002_02503_gb300 import fields

    D = 2 if a.lattice == "D2Q9" else 3
    dims = tuple(a.dims)
    if D == 3:
        return fields.taylor_green_3d(dims, a.u0, LATTICE_T0[a.lattice])
    return fields.taylor_green_2d(dims, a.u0, LATTICE_T0[a.lattice], D=2)


# ------------------------------------------------------------------ CPU oracle timing
def oracle_sample(a, seconds):
    """Time the FP64 oracle on a sub-lattice of the workload (same lattice, K, tau)."""
    import oracle
    from paper_2002_02503_gb300 import fields

    nthreads = oracle.default_threads()
    side = 64 if a.lattice != "D3Q39" else 48
    dims = (side, side, side) if a.lattice != "D2Q9" else (256, 256, 1)
    D = 2 if a.lattice == "D2Q9" else 3
    if D == 3:
        rho, u = fields.taylor_green_3d(dims, a.u0, LATTICE_T0[a.lattice])
    else:
        rho, u = fields.taylor_green_2d(dims, a.u0, LATTICE_T0[a.lattice], D=2)
    f = oracle.init_eq(a.lattice, a.K, dims, rho, u)
    C = int(np.prod(dims))
    t0 = time.perf_counter()
    f = oracle.run(a.lattice, a.K, a.tau, dims, f, 1, nthreads)
    one = time.perf_counter() - t0
    steps = int(max(1, min(200, seconds / max(one, 1e-6))))
    t0 = time.perf_counter()
    oracle.run(a.lattice, a.K, a.tau, dims, f, steps, nthreads)
    dt = time.perf_counter() - t0
    # the same sub-lattice on one core, for a few steps
    steps1 = int(max(1, min(steps, 0.25 * seconds / max(one * nthreads, 1e-6))))
    t0 = time.perf_counter()
    oracle.run(a.lattice, a.K, a.tau, dims, f, steps1, 1)
    dt1 = time.perf_counter() - t0
    return {"value": C * steps / dt / 1e6, "unit": "MLUPS", "cores": nthreads, "kind": "oracle",
            "sample": "%s K=%d tau=%g Taylor-Green sub-lattice %dx%dx%d, %d steps, %.1f s" % (
                a.lattice, a.K, a.tau, dims[0], dims[1], dims[2], steps, dt),
            "single_core": {"value": C * steps1 / dt1 / 1e6, "unit": "MLUPS", "cores": 1,
                            "sample": "the same sub-lattice, %d steps, %.1f s" % (steps1, dt1)}}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.active = False

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            if self.active:
                self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm = []
        mx = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ roofline helpers
def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        p = os.path.join(ROOT, "paper_2002_02503_gb300", "csrc", f)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(a, variant, cpt):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    key = "%s_%dx%dx%d_%s_K%d_v%d_c%d" % (a.lattice, a.dims[0], a.dims[1], a.dims[2], a.storage, a.K, variant, cpt)
    r = rec.get(key)
    if not r or r.get("kernel_hash") != kernel_hash():
        return None
    return r.get("bytes_per_launch")


# ------------------------------------------------------------------ whole-job figures
def combine_ranks(ms, e2e_value, world, device):
    """Independent replicas, one lattice per rank: the job's timed-region time is the slowest
    rank's (max over ranks), and its end-to-end rate is world x the slowest rank's rate."""
    if world == 1:
        return ms, e2e_value
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms, -(e2e_value if e2e_value is not None else 0.0)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_job = -float(t[1]) * world if e2e_value is not None else None
    return float(t[0]), e2e_job


def job_mlups(cells_per_rank, steps, world, t_max_ms):
    """Whole-job million lattice-cell updates per second."""
    return world * cells_per_rank * steps / (t_max_ms / 1e3) / 1e6


# ------------------------------------------------------------------ main arms
def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cpu = oracle_sample(a, a.cpu_seconds)
    out = {"metric": "MLUPS", "value": cpu["value"], "unit": "MLUPS", "n_gpus": a.gpus, "steps": a.steps,
           "warmup": a.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic (Taylor-Green initial field)", "impl": "reference",
           "config": config_of(a), "cpu_baseline": cpu,
           "e2e": {"value": cpu["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def run_ours(a):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2002_02503_gb300 import lbm

    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream(dev)
    dims = tuple(a.dims)
    C = int(np.prod(dims))
    Q = LATTICE_Q[a.lattice]
    rho, u = initial_fields(a)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        s = lbm.Solver(a.lattice, dims, a.tau, a.K, a.storage, stream=stream,
                       storage_range=a.storage_range if a.storage == "q16" else None)
        s.set_fields(rho, u)
        tuned_us = None
        if a.variant is None:
            tuned_us = lbm.lbm_autotune(s.handle, 20)
        else:
            lbm.lbm_set_kernel(s.handle, a.variant, a.cpt or 0, a.block or 0)
        variant, cpt, block = lbm.lbm_get_kernel(s.handle)
        s.set_fields(rho, u)
        s.step(a.warmup)
        barrier()

        clocks = ClockSampler(dev)
        clocks.start()
        time.sleep(0.3)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        clocks.active = True
        ev0.record(stream)
        s.step(a.steps)
        ev1.record(stream)
        ev1.synchronize()
        clocks.active = False
        ms = ev0.elapsed_time(ev1)
        barrier()
        cons = s.conservation()

        # end to end through the C-ABI with host buffers: fields in, K steps, moments out
        e2e = None
        if not a.no_e2e:
            D = 2 if a.lattice == "D2Q9" else 3
            rho_h = torch.from_numpy(rho).pin_memory()
            u_h = torch.from_numpy(np.ascontiguousarray(u)).pin_memory()
            rho_o = torch.empty(C, dtype=torch.float64).pin_memory()
            u_o = torch.empty((D, C), dtype=torch.float64).pin_memory()
            barrier()
            t0 = time.perf_counter()
            lbm.lbm_set_fields(s.handle, rho_h, u_h)
            lbm.lbm_step(s.handle, a.steps)
            lbm.lbm_get_moments(s.handle, rho_o, u_o)
            t_e2e = time.perf_counter() - t0
            barrier()
            h2d = (rho_h.numel() + u_h.numel()) * 8
            d2h = (rho_o.numel() + u_o.numel()) * 8
            e2e = {"value": C * a.steps / t_e2e / 1e6, "unit": "MLUPS",
                   "h2d_bytes_per_step": h2d / a.steps, "d2h_bytes_per_step": d2h / a.steps,
                   "note": "one solve: set_fields from pinned host, %d steps, get_moments to pinned host; "
                           "copies amortised over the steps" % a.steps}
        s.close()
    clocks.stop()

    t_max, e2e_job = combine_ranks(ms, e2e["value"] if e2e is not None else None, world, "cuda")
    if e2e is not None:
        e2e["value"] = e2e_job
    value = job_mlups(C, a.steps, world, t_max)
    if rank == 0:
        bpu = 2 * Q * STORE_BYTES[a.storage]
        per_launch_s = (ms / 1e3) / a.steps
        achieved = bpu * C / per_launch_s / 1e9
        peak, peak_kind = measured_peak()
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": recorded_traffic(a, variant, cpt), "peak_kind": peak_kind,
                "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                "algorithmic_bytes_per_launch": bpu * C,
                "kernel": "step_%s" % {0: "direct", 1: "staged", 2: "pair"}.get(variant, "direct")}
        cpu = None
        if not a.no_cpu_baseline:
            cpu = oracle_sample(a, a.cpu_seconds)
        extras = {}
        if a.precision_report:
            with torch.cuda.stream(stream):
                extras["precision"] = precision_report(stream)
        if not a.no_extras:
            with torch.cuda.stream(stream):
                extras["per_lattice"] = [measure_lattice(*cfg, a.extra_steps, stream) for cfg in PER_LATTICE]
                extras["per_mode"] = [measure_lattice(*cfg[:6], a.extra_steps, stream, model=cfg[6], theta=cfg[7],
                                                      field=cfg[8] if len(cfg) > 8 else None)
                                      for cfg in PER_MODE]
            from paper_2002_02503_gb300 import serve

            peak, _ = measured_peak()
            extras["batched"] = []
            for storage in ("f32", "f16"):
                r = serve.batched_rate(40, a.extra_steps, storage)
                r["frac_of_measured_hbm"] = r["MLUPS"] * 1e6 * r["bytes_per_update"] / 1e9 / peak
                extras["batched"].append(r)
            if a.serve > 0:

                trace = serve.make_trace(a.serve, rate=a.serve_rate)
                pool_stats, _ = serve.serve_pool(trace)
                pool16_stats, _ = serve.serve_pool(trace, storage="f16")
                poolq_stats, _ = serve.serve_pool(trace, storage="q16", storage_range=0.0)
                plain_stats, _ = serve.serve_plain(trace)
                # capacity: the same requests all arriving at once
                burst = [dict(r, arrival=0.0) for r in trace]
                burst_pool, _ = serve.serve_pool(burst)
                burst_poolq, _ = serve.serve_pool(burst, storage="q16", storage_range=0.0)
                burst_plain, _ = serve.serve_plain(burst)
                extras["serving_accuracy"] = serve.served_accuracy()
                extras["serving"] = {
                    "workload": "%d D3Q19 Taylor-Green solves, side log-uniform 32-128, tau U[0.52,1], "
                                "u0 U[0.01,0.08], 100-2000 steps, Poisson %g/s, FP32, K=3" % (a.serve, a.serve_rate),
                    "pool": pool_stats, "pool_f16_storage": pool16_stats,
                    "pool_q16_storage_per_request_range": poolq_stats, "plain_fifo": plain_stats,
                    "capacity_all_at_once": {"pool": burst_pool, "pool_q16_storage_per_request_range": burst_poolq,
                                             "plain_fifo": burst_plain}}
        out = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": a.steps,
               "warmup": a.warmup, "ms_per_step": t_max / a.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": DTYPE_NAME[a.storage], "data": "synthetic (Taylor-Green initial field)",
               "config": config_of(a, {"kernel": {"variant": variant, "cells_per_thread": cpt, "block": block,
                                                  "autotuned_us": tuned_us}}),
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": a.steps,
               "clocks": clocks.summary(),
               "conservation": {"mass": cons[0], "momentum": list(cons[1:])}}
        out.update(extras)
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
