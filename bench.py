#!/usr/bin/env python3
"""RK3 cell-updates/s of the GB300 dycore (one JSON line on rank 0).

Workload (default): the 3D warm bubble over a Gaussian hill, 256 x 256 x 128 cells, dx = dy = 50 m,
stretched dz from 20 m, FP64, WENO5 scalars, upwind-5 momenta, 6 acoustic substeps (10 substep
passes per step).  A step is one RK3 step (3 stages, slow tendencies + substeps).  Inputs are
resident in HBM; the working set (~2.7 GB) is far larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (under torchrun): independent replicas, one per GPU (the dycore runs one domain per GPU),
value = total cell-updates over all ranks / max-over-ranks time.  --shard runs the x-y pencil
decomposition instead (weak-scaled: one benchmark-sized interior per rank, halo exchange per step;
on one GPU, --shard-ranks P pencils share it).
--impl reference times the FP64 CPU oracle on the host cores on a bounded sample of the same
workload (the method's reference implementation here is that oracle).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RK3 cell-updates/s"
UNIT = "cell-updates/s"

# Algorithmic HBM words (FP64) per unit and FP64 flops per unit of each kernel: the ideal traffic
# if every input is read once and every output written once, and the floating-point operations
# of the formulas (FMA = 2).  unit: "cell" (nx*ny*nz) or "wface" (nx*ny*(nz+1)).
KERNEL_MODEL = {
    "flux_theta":  {"unit": "wface", "words": 7, "flops": 210},
    "sub_expl":    {"unit": "cell", "words": 20, "flops": 56},
    "sub_col":     {"unit": "cell", "words": 11, "flops": 12},
    "sub_fin":     {"unit": "cell", "words": 10, "flops": 18},
    "sub_horiz":   {"unit": "cell", "words": 10, "flops": 30},
    "flux_u":      {"unit": "wface", "words": 7, "flops": 63},
    "flux_v":      {"unit": "wface", "words": 7, "flops": 63},
    "flux_w":      {"unit": "wface", "words": 7, "flops": 63},
    "rhs_cells":   {"unit": "cell", "words": 6, "flops": 20},
    "rhs_u":       {"unit": "cell", "words": 6, "flops": 25},
    "rhs_v":       {"unit": "cell", "words": 6, "flops": 25},
    "rhs_w":       {"unit": "wface", "words": 7, "flops": 25},
    "stage_begin": {"unit": "wface", "words": 20, "flops": 60},
    "prep":        {"unit": "wface", "words": 10, "flops": 40},
    "tri_build":   {"unit": "cell", "words": 14, "flops": 90},
    "stage_end":   {"unit": "wface", "words": 15, "flops": 5},
    "wall_bc":     {"unit": "none", "words": 0, "flops": 0},
    # moist path: Kessler reads rho, rho theta, 3 water species, writes 4 (pow/exp/sqrt each ~20 flop)
    "kessler_fall": {"unit": "cell", "words": 3, "flops": 40},
    "kessler":     {"unit": "cell", "words": 11, "flops": 200},
    "moist_diff":  {"unit": "cell", "words": 8, "flops": 90},
    "relax":       {"unit": "wface", "words": 18, "flops": 30},
    "tke_diff":    {"unit": "cell", "words": 4, "flops": 40},
    "tke_update":  {"unit": "cell", "words": 5, "flops": 12},
    "tracer_update": {"unit": "cell", "words": 5, "flops": 10},
    "tracer_flux": {"unit": "wface", "words": 10, "flops": 210},
    # anelastic projection: complex FP64 field in and out per pass; an FFT of length n costs
    # 5 log2 n flops per point (forward x + y, or inverse y + x, in one scope)
    "anel_fft":    {"unit": "cell", "words": 8, "flops": 80},
    "anel_tri":    {"unit": "cell", "words": 6, "flops": 14},
    "anel_div":    {"unit": "cell", "words": 5, "flops": 8},
    "anel_correct": {"unit": "wface", "words": 9, "flops": 10},
    "anel_stage":  {"unit": "wface", "words": 12, "flops": 16},
    "anel_begin":  {"unit": "cell", "words": 4, "flops": 2},
}
# DRAM bytes per unit from an ncu capture of the kernel as it stands (dram__bytes_read.sum +
# dram__bytes_write.sum of a 128^3 hill-bubble launch / its units; profiles/ has the summary),
# scaled to the benchmark's units.  A kernel missing here reports traffic null.
KERNEL_TRAFFIC_PER_UNIT = {"flux_theta": 39.9, "sub_expl": 160.8}
# the same for the FP32-perturbation kernels: DRAM bytes per cell of one launch of the column sweep
# in a 384 x 384 x 160 convective-ABL capture (2.232 GB over 23.6 M cells; traffic grows with the
# cells); kernels changed since their capture are left out (traffic null)
KERNEL_TRAFFIC_PER_UNIT_MIXED = {"mx_sub_vert": 94.6}
# mixed path: algorithmic bytes per cell per launch (FP32 fields, FP64 LU factors and d');
# these kernels are bound by HBM or latency, so their roofline is in GB/s
KERNEL_MODEL_MIXED = {
    "mx_sub_vert":    {"unit": "cell", "bytes": 92},
    "mx_sub_col":     {"unit": "cell", "bytes": 68},
    "mx_sub_expl":    {"unit": "cell", "bytes": 52},
    "mx_sub_fin":     {"unit": "cell", "bytes": 32},
    "mx_sub_horiz":   {"unit": "cell", "bytes": 32},
    "mx_closure_mlp": {"unit": "cell", "bytes": 56},
    "mx_cl_edges":    {"unit": "wface", "bytes": 24},
    "mx_cl_div":      {"unit": "wface", "bytes": 68},
    "mx_sgs_edges":   {"unit": "wface", "bytes": 24},
    "mx_sgs_mu":      {"unit": "cell", "bytes": 44},
    "mx_sgs_tau":     {"unit": "wface", "bytes": 28},
    "mx_sgs_div":     {"unit": "wface", "bytes": 64},
    "mx_flux_theta":  {"unit": "wface", "bytes": 28},
    "mx_flux_u":      {"unit": "wface", "bytes": 28},
    "mx_flux_v":      {"unit": "wface", "bytes": 28},
    "mx_flux_w":      {"unit": "wface", "bytes": 28},
    "mx_rhs_cells":   {"unit": "cell", "bytes": 32},
    "mx_rhs_u":       {"unit": "cell", "bytes": 28},
    "mx_rhs_v":       {"unit": "cell", "bytes": 28},
    "mx_rhs_w":       {"unit": "wface", "bytes": 24},
    "mx_tri_build":   {"unit": "cell", "bytes": 44},
    "mx_stage_begin": {"unit": "wface", "bytes": 96},   # with the face velocities and mass fluxes
    "mx_prep":        {"unit": "wface", "bytes": 36},
    "mx_stage_end":   {"unit": "wface", "bytes": 60},
}
# FP64 peak from the unit count ncu reports on GB300 (sm__sass_thread_inst_executed_op_dfma_
# pred_on.sum.peak_sustained = 304 per cycle, 2 per SM) x 2 flop x 2.07 GHz maximum SM clock
FP64_PEAK_TFLOPS = 304 * 2 * 2.07e9 / 1e12


def step_bytes_per_cell_update(precision, n_substeps):
    """Algorithmic HBM bytes of one whole RK3 step per cell (each kernel reads its inputs once
    and writes its outputs once, stage init/finalize folded into the first/last substep):
    3 stages x (10 words of slow tendencies + 10 of stage init/finalize) + 17 words per substep
    pass, sum over stages of the substep counts = 1 + ns/2 + ns.  FP64: 8-byte words; the
    FP32-perturbation form: 950 B at ns = 6 and 1400 B at ns = 10 (FP32 fields, FP64 tridiagonal
    coefficients)."""
    passes = 1 + n_substeps // 2 + n_substeps
    if precision == "fp64":
        return 8 * (60 + 17 * passes)
    return {6: 950.0, 10: 1400.0}.get(n_substeps, 4.0 * (60 + 17 * passes) + 12.0 * passes)


def kernel_roofline(name, tms, nl, total, wl, hbm, hsrc):
    """Roofline object of one kernel from its profiled time: HBM-bound kernels (the FP32 path)
    in GB/s of algorithmic bytes, FP64-ALU-bound kernels in TFLOP/s of algorithmic flops."""
    avg_s = tms / nl * 1e-3
    units_of = {"cell": wl.ncell, "wface": wl.nx * wl.ny * (wl.nz + 1), "none": 0}
    if name in KERNEL_MODEL_MIXED:
        mm = KERNEL_MODEL_MIXED[name]
        units = units_of[mm["unit"]]
        gbs = mm["bytes"] * units / avg_s / 1e9
        tpu = KERNEL_TRAFFIC_PER_UNIT_MIXED.get(name)
        return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "traffic": None if tpu is None else tpu * units, "kernel": name,
                "alg_bytes": mm["bytes"] * units, "kernel_avg_ms": tms / nl,
                "kernel_share": tms / total, "peak_source": hsrc}
    model = KERNEL_MODEL.get(name, {"unit": "cell", "words": 0, "flops": 0})
    units = units_of[model["unit"]]
    flops = model["flops"] * units
    bytes_ = 8 * model["words"] * units
    fp64_tf = flops / avg_s / 1e12
    hbm_gbs = bytes_ / avg_s / 1e9
    tpu = KERNEL_TRAFFIC_PER_UNIT.get(name)
    return {"bound": "alu", "achieved": fp64_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": fp64_tf / FP64_PEAK_TFLOPS, "traffic": None if tpu is None else tpu * units,
            "kernel": name, "alg_flops": flops, "kernel_avg_ms": tms / nl, "kernel_share": tms / total,
            "peak_source": "derived: 304 DFMA/cycle (ncu unit count) x 2 flop x 2.07 GHz",
            "hbm": {"achieved": hbm_gbs, "peak": hbm, "unit": "GB/s", "frac": hbm_gbs / hbm,
                    "peak_source": hsrc}}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured", d
    return 6800.0, "fallback", {}


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        try:
            for line in open(self.f.name):
                t = [x.strip() for x in line.split(",")]
                if len(t) >= 9:
                    rows.append(t)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.f.name)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(n_gpus, backend="nccl"):
    """torchrun environment -> (world size, rank, local rank, process group or None).  The GPU run
    uses NCCL; the CPU tests of the replica coordination use gloo."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return ws, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v, device="cuda"):
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def replica_value(pg, ws, units_per_rank, seconds, device="cuda"):
    """Whole-job throughput of N independent replicas: all ranks' units over the slowest rank's
    time (weak scaling: each rank runs the full workload)."""
    t = max_over_ranks(pg, seconds, device)
    return ws * units_per_rank / t, t


def oracle_rate(wl_sample, steps, threads=None):
    """Cell-updates/s of the FP64 oracle on a workload sample (host cores); returns
    (rate, seconds, threads used)."""
    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from conftest import make_oracle
    used = oracle.set_threads(threads or os.cpu_count() or 1)
    o = make_oracle(wl_sample)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return wl_sample.ncell * steps / dt, dt, used


def workload(args):
    from paper_2412_04395_gb300 import workloads as W
    prec = W.PREC_MIXED32 if args.precision == "mixed" else W.PREC_FP64
    if args.case == "hill_bubble":
        if args.precision != "fp64":
            raise SystemExit("the hill bubble runs over terrain, which the mixed path does not support")
        if args.grid:
            return W.hill_bubble(nx=args.grid[0], ny=args.grid[1], nz=args.grid[2])
        return W.hill_bubble()
    if args.case == "density_current":
        return W.density_current().with_(precision=prec)
    if args.case == "convective_abl":
        nx, ny, nz = args.grid or (512, 512, 160)
        wl = W.convective_abl(nx=nx, ny=ny, nz=nz, dx=40.0).with_(precision=prec)
        if args.closure == "learned":
            wl = wl.with_(closure=W.CLOSURE_LEARNED)
        return wl
    if args.case == "neutral_abl":
        nx, ny, nz = args.grid or (1024, 1024, 128)
        return W.neutral_abl(nx=nx, ny=ny, nz=nz, dx=10.0).with_(precision=prec)
    if args.case == "paper_scaling":
        nx, ny, nz = args.grid or (512, 512, 256)
        return W.paper_scaling(nx=nx, ny=ny, nz=nz).with_(precision=prec)
    raise SystemExit(f"unknown case {args.case}")


def sample_workload(args):
    """Bounded sample of the benchmark workload for the CPU oracle: same spacing, stretching,
    hill, bubble and physics on a 64 x 64 horizontal window (the hill scaled to the window)."""
    from paper_2412_04395_gb300 import workloads as W
    if args.case == "hill_bubble":
        return W.hill_bubble(nx=64, ny=64, nz=128, dx=50.0)
    if args.case == "convective_abl":
        return W.convective_abl(nx=32, ny=32, nz=160, dx=40.0).with_(precision=W.PREC_FP64)
    return W.density_current(nx=64, ny=4, nz=64)


def run_reference(args):
    ws, rank, local, pg = dist_setup(args.gpus)
    if rank != 0:
        return
    from paper_2412_04395_gb300 import workloads as W  # noqa: F401
    import oracle
    oracle.build_oracle()
    wl = workload(args)
    sw = sample_workload(args)
    for _ in range(args.warmup):
        oracle_rate(sw, 1)
    t = 0.0
    for _ in range(args.steps):
        _, dt, used = oracle_rate(sw, 1)
        t += dt
    v = sw.ncell * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "grid": [wl.nx, wl.ny, wl.nz], "sample_grid": [sw.nx, sw.ny, sw.nz]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": f"{sw.nx}x{sw.ny}x{sw.nz} window of {wl.name}, 1 step per timed step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_steps(d, steps, warmup):
    """Device time (ms) of `steps` graph-launched steps after `warmup`, CUDA events on the bound stream."""
    import torch
    d.erf_rk3_step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(d.stream)
    d.erf_rk3_step(steps)
    e1.record(d.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def closure_blob(wl, d):
    """The trained closure blob shipped with the package if present, else random weights with
    statistics from the initial state (throughput only)."""
    path = os.path.join(ROOT, "paper_2412_04395_gb300", "data", "closure_convective_abl.bin")
    if os.path.exists(path):
        return open(path, "rb").read(), "trained"
    rng = np.random.default_rng(0)
    feats = d.erf_closure_features().cpu().numpy().astype(np.float64)
    mu, sd = feats.mean(axis=0), feats.std(axis=0)
    sd = np.where(sd > 0, sd, 1.0)
    parts = [mu, sd, np.zeros(9), np.full(9, 0.01)]
    for a, b in zip((12, 64, 64, 64), (64, 64, 64, 9)):
        parts += [rng.normal(size=a * b) * np.sqrt(1.0 / a), np.zeros(b)]
    body = np.concatenate(parts).astype(np.float32)
    return np.array([0x4D465245, 1], dtype=np.uint32).tobytes() + body.tobytes(), "random"


def _e2e_rate(d, wl, steps, dtype):
    """Cell-updates/s end to end through the C ABI with pinned host buffers: every step uploads
    the five state fields from the host, advances one step and downloads them (dtype "f64" or
    "f32" host buffers; the library converts on the device).  Returns the e2e object."""
    import torch
    from paper_2412_04395_gb300.erf import FIELDS
    tdt = torch.float64 if dtype == "f64" else torch.float32
    code = 0 if dtype == "f64" else 1
    host = {k: torch.empty(d._shape(k), dtype=tdt).pin_memory() for k in
            ("rho", "rhotheta", "rhou", "rhov", "rhow")}
    L = d.L
    for k, t in host.items():
        assert L.erf_get_state(d.h, FIELDS[k], t.data_ptr(), 0, code) == 0
    nbytes = sum(t.numel() * t.element_size() for t in host.values())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        for k, t in host.items():
            st = L.erf_set_state(d.h, FIELDS[k], t.data_ptr(), 0, code)
            assert st == 0
        d.erf_rk3_step(1)
        for k, t in host.items():
            st = L.erf_get_state(d.h, FIELDS[k], t.data_ptr(), 0, code)
            assert st == 0
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    del host
    return {"value": wl.ncell * steps / te, "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "steps": steps, "host_dtype": dtype}


def _time_form(wl, steps, out, name, prec, e2e_steps=0):
    """Cell-updates/s of one form of a workload (CUDA events around graph-launched steps after
    3 warm-up steps), its per-kernel device times over one further step, the roofline of its
    dominant kernel, its step-level fraction of the HBM roofline (cell-updates/s x the step's
    algorithmic bytes per cell-update / measured HBM bandwidth) and, with e2e_steps, its rate end
    to end through the C ABI with host buffers."""
    import torch
    from paper_2412_04395_gb300 import workloads as W
    from paper_2412_04395_gb300.erf import Dycore
    d = Dycore(wl)
    if wl.moist:
        d.erf_set_initial_moist(wl.dtheta, wl.qv, wl.u, wl.v, wl.w)
    else:
        d.erf_set_initial(wl.dtheta, wl.u, wl.v, wl.w)
    if wl.closure == W.CLOSURE_DEARDORFF and wl.tke is not None:
        d.erf_set_state("rhotke", d.erf_get_state("rho") * wl.tke)
    if wl.closure == W.CLOSURE_LEARNED:
        blob, kind = closure_blob(wl, d)
        d.erf_set_closure_weights(blob)
        out["learned_weights"] = kind
    ms = time_steps(d, steps, 3)
    prof = d.erf_profile_steps(1)
    total = sum(v[0] for v in prof.values())
    top_name, (tms, nl) = max(prof.items(), key=lambda kv: kv[1][0])
    hbm, hsrc, _ = peaks()
    value = wl.ncell * steps / (ms * 1e-3)
    sb = step_bytes_per_cell_update(prec, wl.n_substeps)
    rec = {"value": value, "ms_per_step": ms / steps, "steps": steps,
           "roofline": kernel_roofline(top_name, tms, nl, total, wl, hbm, hsrc),
           "hbm_frac_step": value * sb / (hbm * 1e9), "step_alg_bytes_per_cell_update": sb,
           "kernel_ms_per_step": {k: round(v[0], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])[:10]},
           "kernel_share": {k: round(v[0] / total, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])[:10]}}
    if e2e_steps > 0:
        rec["e2e"] = _e2e_rate(d, wl, e2e_steps, "f32" if prec == "mixed" else "f64")
    out[name] = rec
    d.close()
    del d
    torch.cuda.empty_cache()


def precision_comparison(args):
    """FP64 Smagorinsky vs FP32 perturbations (Smagorinsky) vs FP32 + learned closure (BF16
    tensor-core inference), each timed alone on the same GB300: the coarse convective ABL
    (default 2048 x 2048 x 160 at 40 m, 671 M cells), the neutral ABL 1024 x 1024 x 128 at 10 m
    and, as context, the paper's scaling workload 512 x 512 x 256 at 4 m with upwind-3 (FP64 vs
    FP32)."""
    from paper_2412_04395_gb300 import workloads as W
    nx, ny, nz = args.cmp_grid
    base = W.convective_abl(nx=nx, ny=ny, nz=nz, dx=40.0)
    out = {"workload": f"convective_abl {nx}x{ny}x{nz} at 40 m, ns=10, Smagorinsky/learned, MOST"}
    fp64_steps = max(1, args.cmp_steps // 4)
    _time_form(base.with_(precision=W.PREC_FP64), fp64_steps, out, "fp64_smagorinsky", "fp64")
    _time_form(base.with_(precision=W.PREC_MIXED32), args.cmp_steps, out, "fp32_smagorinsky", "mixed")
    _time_form(base.with_(precision=W.PREC_MIXED32, closure=W.CLOSURE_LEARNED), args.cmp_steps, out,
               "fp32_learned", "mixed", e2e_steps=args.cmp_e2e_steps)
    del base
    out["fp32_learned_over_fp64"] = out["fp32_learned"]["value"] / out["fp64_smagorinsky"]["value"]
    out["fp32_over_fp64"] = out["fp32_smagorinsky"]["value"] / out["fp64_smagorinsky"]["value"]
    if args.neutral_grid[0] > 0:
        mx, my, mz = args.neutral_grid
        nb = W.neutral_abl(nx=mx, ny=my, nz=mz, dx=10.0)
        neu = {"workload": f"neutral_abl {mx}x{my}x{mz} at 10 m, ns=10, Smagorinsky, MOST"}
        _time_form(nb.with_(precision=W.PREC_FP64), fp64_steps, neu, "fp64", "fp64")
        _time_form(nb.with_(precision=W.PREC_MIXED32), args.cmp_steps, neu, "fp32", "mixed")
        neu["fp32_over_fp64"] = neu["fp32"]["value"] / neu["fp64"]["value"]
        out["neutral_abl"] = neu
    if args.paper_grid[0] > 0:
        # context: the paper's scaling workload (Sec. 5.2), upwind-3 + Smagorinsky at 4 m
        px, py, pz = args.paper_grid
        pw = W.paper_scaling(nx=px, ny=py, nz=pz)
        pap = {"workload": f"paper_scaling {px}x{py}x{pz} at 4 m, upwind-3, ns=10, Smagorinsky, MOST"}
        _time_form(pw.with_(precision=W.PREC_FP64), fp64_steps, pap, "fp64", "fp64")
        _time_form(pw.with_(precision=W.PREC_MIXED32), args.cmp_steps, pap, "fp32", "mixed")
        pap["fp32_over_fp64"] = pap["fp32"]["value"] / pap["fp64"]["value"]
        out["paper_scaling"] = pap
    return out


def extension_lines(args):
    """Cell-updates/s of the paths beyond the RK3 dycore (CUDA events around graph-launched steps
    after 3 warm-up steps, per-kernel times of one further step), each on one GB300:
      * the moist squall line (Sec. 4.1.3) at its full size, 1500 x 4 x 240 at 100 m, FP64, Kessler
        microphysics, constant nu = alpha = 200 m^2/s, relaxation-zone open boundaries;
      * the Deardorff 1.5-order closure (FP64) on the convective ABL at 512 x 512 x 160 (40 m);
      * the anelastic equation set (SSP-RK2 + FFT projection, FP64) on a 3D warm bubble,
        256 x 256 x 128 at 50 m."""
    from paper_2412_04395_gb300 import workloads as W
    out = {}
    sq = W.squall_line()
    _time_form(sq, args.ext_steps, out, "squall_line_fp64_kessler", "fp64")
    out["squall_line_fp64_kessler"]["workload"] = "squall_line 1500x4x240 at 100 m, dt 0.25 s, ns 6"
    cb = W.convective_abl(nx=512, ny=512, nz=160, dx=40.0).with_(precision=W.PREC_FP64,
                                                                closure=W.CLOSURE_DEARDORFF, Pr_t=1.0 / 3.0)
    zc = 0.5 * (cb.zeta[:-1] + cb.zeta[1:])
    cb = cb.with_(tke=np.broadcast_to((0.5 * np.exp(-zc / 400.0) + 0.01)[:, None, None], (cb.nz, cb.ny, cb.nx)).copy())
    _time_form(cb, max(1, args.ext_steps // 2), out, "convective_abl_fp64_deardorff", "fp64")
    out["convective_abl_fp64_deardorff"]["workload"] = "convective_abl 512x512x160 at 40 m, Deardorff, ns 10"
    zeta = W.uniform_zeta(128, 50.0)
    X, Y, Z = W.cell_coords(256, 256, zeta, 50.0, 50.0)
    r = np.sqrt((X - 6400.0) ** 2 + (Y - 6400.0) ** 2 + (Z - 1500.0) ** 2) / 1000.0
    an = W.Workload("anelastic_bubble", 256, 256, 128, 50.0, 50.0, zeta, dt=1.0, closure=W.CLOSURE_NONE,
                    dtheta=np.where(r < 1.0, 2.0 * np.cos(0.5 * np.pi * r) ** 2, 0.0), anelastic=1)
    _time_form(an, args.ext_steps, out, "anelastic_bubble_fp64", "fp64")
    out["anelastic_bubble_fp64"]["workload"] = "anelastic warm bubble 256x256x128 at 50 m, SSP-RK2 + FFT projection"
    return out


def run_ours(args):
    import torch
    ws, rank, local, pg = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    from paper_2412_04395_gb300.erf import Dycore, FIELDS
    wl = workload(args)
    d = Dycore(wl, device=f"cuda:{local}")
    d.erf_set_initial(wl.dtheta, wl.u, wl.v, wl.w)
    if args.column_fusion != -1:
        from paper_2412_04395_gb300.erf import ERF_OPT_COLUMN_FUSION
        d.erf_set_option(ERF_OPT_COLUMN_FUSION, args.column_fusion)
    if args.warp_columns != -1:
        from paper_2412_04395_gb300.erf import ERF_OPT_WARP_COLUMNS
        d.erf_set_option(ERF_OPT_WARP_COLUMNS, args.warp_columns)
    if args.closure == "learned":
        blob, _ = closure_blob(wl, d)
        d.erf_set_closure_weights(blob)
    stream = d.stream
    # warm-up (graph capture happens on the first step)
    d.erf_rk3_step(args.warmup)
    torch.cuda.synchronize()
    diag0 = d.erf_diagnostics()
    kps = diag0["kernels_per_step"]
    # timed region: K graph launches, CUDA events on the bound stream
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as cs:
        barrier(pg)
        torch.cuda.synchronize()
        ev0.record(stream)
        d.erf_rk3_step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(pg)
    clocks = cs.summary()
    ms = ev0.elapsed_time(ev1)
    diag = d.erf_diagnostics()
    value, sec = replica_value(pg, ws, wl.ncell * args.steps, ms * 1e-3)
    ms = sec * 1e3

    # per-kernel device times (event-bracketed direct launches of 2 further steps)
    prof = d.erf_profile_steps(2)
    total = sum(v[0] for v in prof.values())
    name, (tms, nl) = max(prof.items(), key=lambda kv: kv[1][0])
    hbm, hsrc, pk = peaks()
    roof = kernel_roofline(name, tms, nl, total, wl, hbm, hsrc)
    sb = step_bytes_per_cell_update(args.precision, wl.n_substeps)
    hbm_frac_step = (value / ws) * sb / (hbm * 1e9)

    # end to end through the C ABI: every step uploads the state from pinned host memory,
    # advances one step and downloads the state
    e2e = None
    if args.e2e_steps > 0:
        e2e = _e2e_rate(d, wl, args.e2e_steps, "f64" if args.precision == "fp64" else "f32")
        te = wl.ncell * args.e2e_steps / e2e["value"]
        te = max_over_ranks(pg, te)
        e2e["value"] = ws * wl.ncell * args.e2e_steps / te

    cmp = None
    if args.cmp_steps > 0:
        d.close()
        del d
        torch.cuda.empty_cache()
        cmp = precision_comparison(args)
    ext = extension_lines(args) if args.ext_steps > 0 else None

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        import oracle
        oracle.build_oracle()
        sw = sample_workload(args)
        v, dt, used = oracle_rate(sw, args.cpu_steps)
        cpu = {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
               "sample": f"{args.cpu_steps} steps of a {sw.nx}x{sw.ny}x{sw.nz} window of {wl.name} "
                         f"({dt:.1f} s on {used} threads)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
                "data": "synthetic",
                "config": {"workload": wl.name, "grid": [wl.nx, wl.ny, wl.nz], "dx": wl.dx,
                           "substeps": wl.n_substeps, "precision": args.precision, "closure": args.closure,
                           "parallelism": f"replicas{ws}", "warp_columns": args.warp_columns,
                           "l2": "working set >> L2 (no flush needed)"},
                "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                           "reasons": clocks["reasons"], "samples": clocks["samples"]},
                "e2e": e2e, "gpu_launches": kps * args.steps, "kernels_per_step": kps,
                "roofline": roof, "cpu_baseline": cpu, "precision_comparison": cmp, "extensions": ext,
                "mass_rel_drift": abs(diag["mass"] - diag0["mass"]) / abs(diag0["mass"]),
                "mass_drift_steps": args.steps,
                "hbm_frac_step": hbm_frac_step, "step_alg_bytes_per_cell_update": sb,
                "kernel_times_ms": {k: round(v[0] / 2, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}}
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def run_sharded(args):
    """The x-y pencil decomposition (decomp.py), weak-scaled: every rank owns an interior of the
    benchmark's horizontal size (the global domain is px x py of them), advances its window (the
    interior plus a halo of one step's reach) and refreshes the halo once per step.  Under
    torchrun (N > 1) one rank per GPU with the halo strips sent point to point (NCCL); on one GPU
    (--shard-ranks P) the P windows are handles on the same GPU and the strips are device copies
    (decomp.LocalRouter), which measures what the decomposition itself costs.  value = interior
    cell-updates of all ranks / the slowest rank's time."""
    import torch
    from paper_2412_04395_gb300 import decomp as D
    from paper_2412_04395_gb300.erf import Dycore
    ws, rank, local, pg = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    P = ws if ws > 1 else max(1, args.shard_ranks)
    px, py = D.shard_grid(P)
    base = workload(args)
    g_args = argparse.Namespace(**vars(args))
    g_args.grid = [base.nx * px, base.ny * py, base.nz]
    wl = workload(g_args)
    dec = D.PencilDecomp(wl.nx, wl.ny, px, py, D.step_reach(wl.n_substeps, wl.terrain is not None))
    mine = [rank] if ws > 1 else list(range(P))
    eng = {}
    for r in mine:
        w = D.window_workload(wl, dec, r)
        eng[r] = Dycore(w, device=f"cuda:{local}")
        eng[r].erf_set_initial(w.dtheta, w.u, w.v, w.w)
    router = D.LocalRouter(dec, [eng[r] for r in range(P)]) if ws == 1 else None

    def step():
        for r in mine:
            eng[r].erf_rk3_step(1)
        if ws > 1:
            D.exchange(dec, rank, eng[rank], pg)
        elif P > 1:
            router.exchange()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    kps = eng[mine[0]].erf_diagnostics()["kernels_per_step"]
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as cs:
        barrier(pg)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(pg)
    clocks = cs.summary()
    sec = max_over_ranks(pg, ev0.elapsed_time(ev1) * 1e-3)
    interior = base.nx * base.ny * base.nz
    value = P * interior * args.steps / sec
    p0 = dec.pencil(mine[0])
    sends, _ = dec.messages(mine[0])
    strip_cols = sum(b[1] * b[3] for _, _, _, b in sends)
    col_bytes = eng[mine[0]].erf_column_block_bytes(1, 1)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
                "data": "synthetic",
                "config": {"workload": f"{wl.name} sharded", "grid": [wl.nx, wl.ny, wl.nz],
                           "interior_per_rank": [base.nx, base.ny, base.nz],
                           "window_per_rank": [p0.nxw, p0.nyw, wl.nz], "halo": dec.halo,
                           "parallelism": f"pencil{px}x{py}" + ("" if ws > 1 else f"-on-1-gpu"),
                           "transport": "nccl point-to-point" if ws > 1 else "device copies (one process)",
                           "l2": "working set >> L2 (no flush needed)"},
                "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                           "reasons": clocks["reasons"], "samples": clocks["samples"]},
                "e2e": None, "gpu_launches": kps * args.steps * len(mine),
                "halo_bytes_per_step_per_rank": strip_cols * col_bytes,
                "redundant_fraction": p0.nxw * p0.nyw / (base.nx * base.ny) - 1.0,
                "roofline": None, "cpu_baseline": None}
        print(json.dumps(line), flush=True)
    for d in eng.values():
        d.close()
    if pg is not None:
        pg.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--case", default="hill_bubble")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=20)
    ap.add_argument("--cmp-grid", type=int, nargs=3, default=[2048, 2048, 160],
                    help="grid of the precision comparison (convective ABL at 40 m)")
    ap.add_argument("--neutral-grid", type=int, nargs=3, default=[1024, 1024, 128],
                    help="grid of the neutral-ABL FP64/FP32 line (0 0 0 skips it)")
    ap.add_argument("--paper-grid", type=int, nargs=3, default=[512, 512, 256],
                    help="grid of the paper's scaling workload (upwind-3) FP64/FP32 line (0 0 0 skips it)")
    ap.add_argument("--cmp-steps", type=int, default=8, help="timed steps per FP32 form (FP64: a quarter); 0 skips")
    ap.add_argument("--cmp-e2e-steps", type=int, default=2,
                    help="steps of the FP32 + learned form timed end to end through the C ABI with host buffers")
    ap.add_argument("--ext-steps", type=int, default=6,
                    help="timed steps of the moist, Deardorff and anelastic lines (0 skips them)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--closure", default="default", choices=["default", "learned"],
                    help="learned: the MLP closure (convective_abl with --precision mixed)")
    ap.add_argument("--grid", type=int, nargs=3, default=None,
                    help="nx ny nz of a smaller window of the workload (profiling runs only)")
    ap.add_argument("--column-fusion", type=int, default=-1, choices=[-1, 0, 1],
                    help="explicit vertical substep part inside the column sweep: -1 by column count")
    ap.add_argument("--shard", action="store_true",
                    help="run the x-y pencil decomposition (one pencil per rank, halo exchange per step)")
    ap.add_argument("--shard-ranks", type=int, default=4,
                    help="with --shard on one GPU: number of pencils emulated there")
    ap.add_argument("--warp-columns", type=int, default=-1, choices=[-1, 0, 1],
                    help="FP64 column kernels one warp per column (1), one thread (0), by column count (-1)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.shard:
        run_sharded(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
