#!/usr/bin/env python3
"""Throughput of the GB300 pressure Poisson solve and the projection step around it.

Metric: Mpts/s per Poisson solve at 512^3, FP32+refine vs FP64, both at relative residual
<= 1e-10.  One step is one pass of the whole hot path over the 512^3 emulsion workload
(200 droplets of density 10 in density 1, triply periodic) with inputs resident in HBM:
set_density (rho0 = min rho, face coefficients), rhs, solve (FP32 transforms + FP64
residual refinement to 1e-10) and correct.  `value` is the solve's rate: grid points over
the CUDA-event time of the solve call inside each step (f in HBM -> p in HBM at the
residual); the whole step's rate is `projection_mpts`.  The FP64 direct solve is timed the
same way and reported beside it (`fp64`), and the other workloads of the same method
(`configs`: the 256^3 and density-ratio-1 emulsions, the 512x512x256 and 1024x1024x512
two-layer boxes) give their solve and projection rates with the error of p against the
FP64 oracle.

  python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference] [--workload NAME]

Prints ONE JSON line on rank 0.  Under torchrun (N > 1) every rank runs an independent
replica of the workload (the single solve has no data-parallel split without an
all-to-all), timing is the max over ranks, value = all ranks' points / that time.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Mpts/s per Poisson solve at 512³: FP32+refine vs FP64 at 1e-10 residual"
GRAPH_MAX_ITER = 3      # FP32 solves at most per graph-capturable refine solve

WORKLOADS = {
    "emulsion512": dict(kind="emulsion", n=512, ratio=10.0,
                        desc="emulsion 512^3 triply periodic, 200 droplets r in [4,12] cells, density ratio 10, "
                             "u** ~ N(0,1), dt = 1e-3"),
    "emulsion512_r1": dict(kind="emulsion", n=512, ratio=1.0,
                           desc="emulsion 512^3 triply periodic, 200 droplets, density ratio 1"),
    "emulsion256": dict(kind="emulsion", n=256, ratio=10.0,
                        desc="emulsion 256^3 triply periodic, 200 droplets, density ratio 10"),
    "two_layer512": dict(kind="two_layer", nx=512, ny=512, nz=256,
                         desc="two-layer 512x512x256, z walls, tanh-stretched dz (beta 1.5), density 1.5 under 1"),
    "two_layer1024": dict(kind="two_layer", nx=1024, ny=1024, nz=512,
                          desc="two-layer 1024x1024x512, z walls, tanh-stretched dz (beta 1.5), density 1.5 "
                               "under 1"),
    "sphere32": dict(kind="sphere", n=32, desc="sphere 32^3 periodic, density 10 in 1"),
}

# Per-kernel algorithmic work per grid point (N = nx ny nz; the half spectrum holds N/2
# complex values, 4 B/point in FP32).  "bound" names the roofline each kernel is held to:
#   hbm: compulsory bytes (each array touched once) / time vs the measured copy bandwidth;
#   alu: FP64 flops (FMA = 2) / time vs the measured FP64 rate.
KERNEL_WORK = {
    # r = f - <f> - L p fused with the forward x transform: reads f, p (FP64), writes the
    # FP32 half spectrum.  On one-spacing grids the defect is an exact fixed-point sum, so
    # few FP64 flops remain and the kernel is held to its compulsory bytes.
    "k_xfwd_residual32": {"bound": "hbm", "bytes": 8 + 8 + 4},
    # the stopping test of the graph-capturable solve: the same defect, norm only
    "k_xres_norm32": {"bound": "hbm", "bytes": 8 + 8},
    "k_xfwd_f32": {"bound": "hbm", "bytes": 8 + 4},
    "k_ycol32": {"bound": "hbm", "bytes": 4 + 4},
    "k_zper32": {"bound": "hbm", "bytes": 4 + 4},
    "k_ztri32": {"bound": "hbm", "bytes": 4 + 4},
    "k_xinv32": {"bound": "hbm", "bytes": 4 + 8},    # first pass: read FP32 spectrum, write p (+ mean of p)
    "k_xinv_acc32": {"bound": "hbm", "bytes": 4 + 16},   # later passes: p += delta (read and write p)
    "k_face_coeffs": {"bound": "hbm", "bytes": None},   # works only in tiles where the density varies
    "k_rho_tiles": {"bound": "hbm", "bytes": 8},
    # the stencils at the compulsory bytes of the method (each input field read once, each
    # output written once): rhs reads u, v, w, rho, p^n, p^{n-1} and writes f; correct reads
    # p, p^n, p^{n-1}, rho, u, v, w and writes u, v, w.  bytes_min: what the kernels move in
    # tiles of constant density, where they skip the density and the extrapolated pressure.
    "k_rhs": {"bound": "hbm", "bytes": 56, "bytes_min": 32},
    "k_correct": {"bound": "hbm", "bytes": 80, "bytes_min": 56, "fp64_instr": 6},   # 3 differences + 3 FMAs
    # momentum predictor (AB2 call): reads u, v, w (FP64) and the M state (3 x 8 B), writes
    # u**, v**, w** and the state; the pre-pass reads u, v, w for max|u|
    "k_momentum": {"bound": "hbm", "bytes": 24 + 24 + 24 + 24},
    "k_mom_umax": {"bound": "hbm", "bytes": 24},
    # FP64 defect with the ends' ghost rules: reads f, p, writes r (neighbours from caches)
    "k_res_ends": {"bound": "hbm", "bytes": 24},
    # VoF step (per split): reconstruction reads phi (halo re-reads from L2) and writes the
    # 32-byte cell record; the flux pass reads the velocity, the upwind record and phi and writes
    # F; the update reads phi, F, the velocity and writes the stage (the final correction, timed
    # with the updates, reads three stages and u, v, w and writes phi: 56 B)
    "k_vof_rec": {"bound": "alu", "bytes": 8 + 32},
    "k_vof_flux": {"bound": "hbm", "bytes": 8 + 32 + 8 + 8},
    "k_vof_update": {"bound": "hbm", "bytes": 32},
}


# On one-spacing grids where the z-marching defect and the register x rows apply, the first FP32
# iterate is held in binary32 until the first update: the first inverse writes 4 B a point
# instead of 8, the first defect and the first update read 4 B of p instead of 8. The first
# defect also writes f's fixed point F - MF (8 B a point), which the norm-only passes read in
# place of f (the same 8 B).
P32_FIRST = {"k_xinv32": 4 + 4, "k_xfwd_residual32": 8 + 4 + 4 + 8, "k_xinv_acc32": 4 + 4 + 8}


def p32_first(c):
    """Whether the plan of case c keeps its first FP32 iterate in binary32."""
    nz, ny, nx = c.shape
    uniform = c.dx == c.dy and all(float(d) == c.dx for d in np.atleast_1d(c.dzf))
    return uniform and nx // 2 in (64, 128, 256, 512) and ny % 8 == 0


def solve_bytes_per_point(k, launches_per_solve, p32):
    """Compulsory bytes per point of one launch of solve kernel k (averaged over its launches in
    one solve: with p32 only the first launch takes the binary32 iterate)."""
    b = KERNEL_WORK[k]["bytes"]
    if not p32 or k not in P32_FIRST or not b:
        return b
    if k == "k_xinv32":
        return P32_FIRST[k]
    n = max(launches_per_solve, 1.0)
    return (P32_FIRST[k] + b * (n - 1.0)) / n


# Kernels of the FP32+refine solve (f -> p); the roofline object names the one that takes most
# of the solve's time.
SOLVE_KERNELS = ("k_xfwd_f32", "k_xfwd_residual32", "k_xres_norm32", "k_ycol32", "k_zper32", "k_ztri32",
                 "k_xinv32", "k_xinv_acc32", "k_finalize")

# DRAM bytes of one launch (dram__bytes_read.sum + dram__bytes_write.sum) from an ncu capture
# of the named workload and kernel.  Only valid for the kernel code that was captured: remove
# the entry when the kernel changes.
MEASURED_TRAFFIC_PER_LAUNCH = {
    # emulsion 512^3, the bench step's third k_correct launch: 5.03 GB read + 3.18 GB written
    # (61.2 B/point; constant-density tiles take 56 B/point, the 11.2 % of tiles with density
    # variation 40 B/point more: 60.5 B/point)
    ("emulsion512", "k_correct"): 5_030_000_000 + 3_180_000_000,
}


def host_info():
    """Host CPU model and core count (for the CPU baseline)."""
    model = None
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                k = line.split(":", 1)
                if len(k) == 2 and k[0].strip() in ("model name", "Model", "CPU part"):
                    model = model or k[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def make_case(name):
    from paper_2204_08834_gb300 import synth
    w = WORKLOADS[name]
    if w["kind"] == "emulsion":
        return synth.emulsion(w["n"], ratio=w["ratio"])
    if w["kind"] == "two_layer":
        return synth.two_layer(w["nx"], w["ny"], w["nz"])
    return synth.sphere(w["n"])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 pipe peak: 499.3 G DFMA lane-ops/s measured on a GB300 by the committed
# micro-benchmark (paper_2204_08834_gb300/microbench/peaks.cu) = 0.999 TFLOP/s with FMA = 2.
FP64_TFLOPS_MEASURED = 0.9986


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to FLUPS_BENCH_CLOCKS_DIR when set (else the temp directory); the
        # JSON line carries their summary
        d = os.environ.get("FLUPS_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"flups_clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def max_over_ranks(values):
    """Element-wise maximum over the ranks of the default process group (the slowest replica
    sets the job time); the identity without a group or with one rank."""
    import torch
    dist = torch.distributed
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_mpts(world, npts, ms):
    """Whole-job throughput of `world` replicas, each processing npts points in ms (weak scaling)."""
    return world * npts / (ms * 1e-3) / 1e6


def timed_steps(plan, c, d0, work, f, p, steps, warmup, rtol, world, graphable=True, final_solve=True):
    """`warmup` + `steps` projections (set_density, rhs, solve, correct) with CUDA events around
    each call on the launch stream; returns the summed times of the timed steps, the FP32
    solves needed, the defect norms and the kernels launched in the timed steps."""
    import torch

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    tot = {"set_density": 0.0, "rhs": 0.0, "solve": 0.0, "correct": 0.0, "step": 0.0}
    iters, rel = [], []
    l0 = None
    for s in range(warmup + steps):
        for k in ("u", "v", "w"):
            work[k].copy_(d0[k])           # restore u** (outside the timed events)
        if s == warmup:
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            l0 = plan.launches
        ev[0].record()
        plan.set_density(d0["rho"])
        ev[1].record()
        plan.rhs(work["u"], work["v"], work["w"], d0["pn"], d0["pnm1"], 2.0, 1.0, c.dt, f)
        ev[2].record()
        # FP32+refine: the graph-capturable form of the solve (the same bits as the
        # host-driven loop; converged iterations exit on the device), so the step has no
        # host round trip; its defect norm is read after the step.  The direct FP64 solve
        # needs no residual evaluation; it is checked after the loop.
        if plan.prec == "fp32_refine" and graphable:
            plan.solve_graphable(f, p, rtol=rtol, max_iter=GRAPH_MAX_ITER)
            info = None
        elif plan.prec == "fp32_refine":
            info = plan.solve(f, p, rtol=rtol, max_iter=12)
        else:
            info = plan.solve(f, p, rtol=0.0, info=False)   # returns None
        ev[3].record()
        plan.correct(p, d0["pn"], d0["pnm1"], 2.0, 1.0, c.dt, work["u"], work["v"], work["w"])
        ev[4].record()
        torch.cuda.synchronize()
        if s >= warmup:
            for q, k in enumerate(("set_density", "rhs", "solve", "correct")):
                tot[k] += ev[q].elapsed_time(ev[q + 1])
            tot["step"] += ev[0].elapsed_time(ev[4])
            if plan.prec == "fp32_refine" and graphable:
                res = plan.solve_result(rtol=rtol)          # defect norm of this step's solve
                rel.append(res.rel_res)
            elif info is not None:
                rel.append(info.rel_res)
    launches = plan.launches - l0
    # FP32 solves actually needed (or, FP64, the residual of the direct solve): one host-driven
    # solve of the same f after the steps, outside the timed region
    if final_solve:
        info = plan.solve(f, p, rtol=rtol, max_iter=12)
        iters.append(info.iters)
        if not rel:
            rel.append(info.rel_res)
    return tot, iters, rel, launches


def measure(c, args, world, fp32_steps, fp64_steps, profile=False, keep=False, clocks=None):
    """FP32+refine and FP64 projections of case `c` through one plan each; per precision the
    step breakdown, solve and projection rates (this rank), defect norms and launches.
    With keep, host copies of f and of both precisions' p; with profile, two more FP32+refine
    steps with the library's per-kernel CUDA events."""
    import torch

    from paper_2204_08834_gb300 import flups

    nz, ny, nx = c.shape
    npts = c.npts
    stream = torch.cuda.current_stream().cuda_stream
    keys = ("u", "v", "w", "rho", "pn", "pnm1")
    d0 = {k: torch.from_numpy(c[k]).cuda() for k in keys}
    work = {k: torch.empty_like(d0["u"]) for k in ("u", "v", "w")}
    f = torch.empty_like(d0["u"])
    p = torch.empty_like(d0["u"])
    torch.cuda.synchronize()
    out = {"npts": npts, "prof": {}}
    for prec, steps in (("fp32_refine", fp32_steps), ("fp64", fp64_steps)):
        with flups.Plan(nx, ny, nz, c.dx, c.dy, c.dzf, c.bc, prec, stream) as plan:
            tot, iters, rel, launches = timed_steps(plan, c, d0, work, f, p, steps, args.warmup, args.rtol, world)
            if profile and prec == "fp32_refine":
                # two more steps with per-kernel CUDA events inside the library (host-driven
                # solve: the kernel sequence of the graph-capturable one without the launches
                # that return at once after convergence, so the per-launch times hold)
                plan.set_profiling(True)
                timed_steps(plan, c, d0, work, f, p, 2, 0, args.rtol, world, graphable=False, final_solve=False)
                out["prof"] = {k: (ms / 2.0, n / 2.0) for k, (ms, n) in plan.profile().items()}
                plan.set_profiling(False)
        torch.cuda.synchronize()      # p: this precision's solution of the step's f (last solve above)
        out[prec] = {"tot": tot, "iters": iters, "rel": rel, "launches": launches, "steps": steps}
        if keep:
            out[prec]["p"] = p.cpu().numpy()
            out["f"] = f.cpu().numpy()
    out["d0"], out["f_dev"] = d0, f
    del work, p
    return out


def rates(m, world):
    """Solve and projection rates (Mpts/s, whole job) of one measure() result."""
    r = {}
    for prec in ("fp32_refine", "fp64"):
        e = m[prec]
        k = e["steps"]
        r[prec] = {"solve_mpts": round(world * m["npts"] / (e["tot"]["solve"] / k * 1e-3) / 1e6, 2),
                   "solve_ms": round(e["tot"]["solve"] / k, 4),
                   "projection_mpts": round(world * m["npts"] / (e["tot"]["step"] / k * 1e-3) / 1e6, 2),
                   "projection_ms": round(e["tot"]["step"] / k, 4),
                   "breakdown_ms": {q: round(v / k, 4) for q, v in e["tot"].items()},
                   "rel_res": max(e["rel"]), "steps": k}
        if prec == "fp32_refine":
            r[prec]["iters"] = statistics.median(e["iters"])
    return r


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_config(name, args, world):
    """One more workload of the method: solve and projection rates of both precisions, and the
    relative L2 error of both p against the FP64 oracle's direct solve of the same f (grids of
    at most 2^27 points; beyond that the oracle's solve does not fit the time budget, and the
    FP32+refine p is compared with the FP64 direct p of the GPU instead)."""
    import torch

    import oracle

    c = make_case(name)
    m = measure(c, args, world, max(3, args.steps // 2), max(2, args.steps // 4), keep=True)
    out = {"workload": WORKLOADS[name]["desc"], "grid": list(c.shape[::-1]), **rates(m, world)}
    p32, p64 = m["fp32_refine"]["p"], m["fp64"]["p"]
    if c.npts <= 1 << 27:
        nz, ny, nx = c.shape
        g = oracle.make_grid(nx, ny, nz, c.dx, c.dy, c.dzf, c.bc)
        po = oracle.solve(m["f"], g, workers=os.cpu_count())
        out["error_vs_oracle"] = {"fp32_refine": rel_err(p32, po), "fp64": rel_err(p64, po),
                                  "definition": "|p - p_oracle|_2 / |p_oracle|_2, same f, oracle = FP64 direct solve"}
    else:
        out["error_vs_oracle"] = {"fp32_refine_vs_fp64_gpu": rel_err(p32, p64),
                                  "definition": "|p_fp32+refine - p_fp64|_2 / |p_fp64|_2 (both GPU, same f); the "
                                                "FP64 direct solve matches the oracle to 1e-11 on every tested grid"}
    del m
    torch.cuda.empty_cache()
    return out


def run_ours(args, rank, world, dev):
    import torch

    from paper_2204_08834_gb300 import flups

    torch.cuda.set_device(dev)
    c = make_case(args.workload)
    nz, ny, nx = c.shape
    npts = c.npts
    stream = torch.cuda.current_stream().cuda_stream
    with ClockSampler(dev) as clk:
        m = measure(c, args, world, args.steps, max(2, args.steps // 2), profile=True, keep=True)
    t32 = m["fp32_refine"]["tot"]["solve"]
    t64 = m["fp64"]["tot"]["solve"]
    s32 = m["fp32_refine"]["tot"]["step"]
    s64 = m["fp64"]["tot"]["step"]
    t32, t64, s32, s64 = max_over_ranks([t32, t64, s32, s64])
    m["fp32_refine"]["tot"]["solve"], m["fp64"]["tot"]["solve"] = t32, t64
    m["fp32_refine"]["tot"]["step"], m["fp64"]["tot"]["step"] = s32, s64
    out = {"c": c, "npts": npts, "m": m, "clocks": clk.summary(), "prof": m["prof"]}
    d0, f = m.pop("d0"), m.pop("f_dev")
    if not args.no_cufft and c.bc == "periodic":
        p = torch.empty_like(f)
        with flups.Plan(nx, ny, nz, c.dx, c.dy, c.dzf, c.bc, "fp64", stream) as plan:
            plan.solve(f, p, rtol=0.0, info=False)
        torch.cuda.synchronize()
        out["cufft"] = cufft_baseline(c, f, p, max(args.steps, 5))
        del p
    del d0, f
    torch.cuda.empty_cache()

    # end to end: the solve through flups_solve_host on pinned host buffers (f in, p out)
    if not args.no_e2e:
        fh = torch.empty(c.shape, dtype=torch.float64, pin_memory=True).numpy()
        np.copyto(fh, m["f"])
        ph = torch.empty(c.shape, dtype=torch.float64, pin_memory=True).numpy()
        e2e_steps = max(1, min(args.steps, 5))
        t_e2e = 0.0
        with flups.Plan(nx, ny, nz, c.dx, c.dy, c.dzf, c.bc, "fp32_refine", stream) as plan:
            for s in range(1 + e2e_steps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                info = plan.solve_host(fh, ph, rtol=args.rtol, max_iter=12)
                t1 = time.perf_counter()
                if s >= 1:
                    t_e2e += t1 - t0
        t_e2e = max_over_ranks([t_e2e])[0]
        out["e2e"] = (t_e2e, e2e_steps, info.rel_res)
        del fh, ph
    if not args.no_ensemble:
        out["ensemble"] = run_ensemble(args)
    if not args.no_learned:
        out["learned"] = run_learned(args)
    if not args.no_momentum:
        out["momentum"] = run_momentum(args)
    if not args.no_ends:
        out["ends"] = run_ends(args)
    if not args.no_vof:
        out["vof"] = run_vof(args)
    out["configs"] = {}
    for name in [q for q in args.configs.split(",") if q]:
        out["configs"][name] = run_config(name, args, world)
    return out


def run_ensemble(args):
    """The mixed-size ensemble: 64 FP32-refine solves of {32, 48, 64, 96, 128}^3 (periodic
    and z walls, density ratios in [1, 20]) as one CUDA graph launch, timed over K replays."""
    import torch

    from paper_2204_08834_gb300 import flups, synth

    cases = [synth.ensemble_member(m) for m in range(64)]
    fs = []
    stream = torch.cuda.current_stream().cuda_stream
    for cm in cases:
        # each member's right-hand side from its own fields by the library's rhs kernel
        d = {k: torch.from_numpy(cm[k]).cuda() for k in ("u", "v", "w", "rho", "pn", "pnm1")}
        f = torch.empty_like(d["u"])
        nz_, ny_, nx_ = cm.shape
        with flups.Plan(nx_, ny_, nz_, cm.dx, cm.dy, cm.dzf, cm.bc, "fp32_refine", stream) as plan:
            plan.set_density(d["rho"])
            plan.rhs(d["u"], d["v"], d["w"], d["pn"], d["pnm1"], 2.0, 1.0, cm.dt, f)
            torch.cuda.synchronize()
        fs.append(f)
    ps = [torch.empty_like(f) for f in fs]
    pts = sum(cm.npts for cm in cases)
    specs = [(cm.shape[2], cm.shape[1], cm.shape[0], cm.dx, cm.dy, cm.dzf, cm.bc) for cm in cases]
    t0 = time.perf_counter()
    with flups.Batch(specs, nstreams=8, autotune=True) as b:
        t_tune = time.perf_counter() - t0
        infos = b.solve(fs, ps, rtol=args.rtol, max_iter=GRAPH_MAX_ITER)   # capture + first launch
        for _ in range(2):
            b.solve(fs, ps, rtol=args.rtol, max_iter=GRAPH_MAX_ITER, info=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            b.solve(fs, ps, rtol=args.rtol, max_iter=GRAPH_MAX_ITER, info=False)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        kernels = b.graph_kernels
    return {"members": len(cases), "points": pts, "ms_per_launch": round(ms, 4),
            "mpts_per_s": round(pts / (ms * 1e-3) / 1e6, 2), "graph_kernels": int(kernels),
            "max_rel_res": max(i.rel_res for i in infos), "autotune_s": round(t_tune, 2),
            "sizes": "{32,48,64,96,128}^3, periodic (even m) / z walls (odd m), density ratio U[1,20]"}


def cufft_baseline(c, f, p_ours, steps):
    """The periodic direct solve with cuFFT (torch.fft: D2Z/Z2D or R2C/C2R over three axes,
    division by the discrete Laplacian's eigenvalues, zero mode set to 0) on the same right-hand
    side, timed with CUDA events like our solve; a reported baseline only (cuFFT is run and
    timed, nothing of it is on the library's path).  Also the largest difference of its FP64 p
    from ours, relative to max |p|."""
    import torch

    if c.bc != "periodic":
        return None
    nz, ny, nx = c.shape
    out = {}
    for name, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        kx = torch.arange(nx // 2 + 1, device="cuda", dtype=torch.float64)
        ky = torch.arange(ny, device="cuda", dtype=torch.float64)
        kz = torch.arange(nz, device="cuda", dtype=torch.float64)
        lam = (-4.0 * torch.sin(torch.pi * kx / nx) ** 2 / c.dx ** 2)[None, None, :] \
            + (-4.0 * torch.sin(torch.pi * ky / ny) ** 2 / c.dy ** 2)[None, :, None] \
            + (-4.0 * torch.sin(torch.pi * kz / nz) ** 2 / c.dzf[0] ** 2)[:, None, None]
        inv = torch.where(lam == 0, torch.zeros_like(lam), 1.0 / lam).to(dt)
        del lam
        fi = f.to(dt)

        def solve():
            return torch.fft.irfftn(torch.fft.rfftn(fi) * inv, s=(nz, ny, nx))

        for _ in range(2):
            pc = solve()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            pc = solve()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        entry = {"ms_per_solve": round(ms, 4), "mpts_per_s": round(c.npts / (ms * 1e-3) / 1e6, 2)}
        if name == "fp64" and p_ours is not None:
            pc = pc - pc.mean()
            entry["max_diff_vs_ours_rel"] = float((pc - p_ours).abs().max() / p_ours.abs().max())
        out[name] = entry
        del pc, fi, inv
        torch.cuda.empty_cache()
    out["kind"] = "cuFFT through torch.fft, periodic direct solve (reported baseline, not on the library path)"
    return out


# Algorithmic flops per grid point of the learned p_hat's convolutions (FMA = 2): 27 taps x
# inputs x outputs x 2 per layer; layer 1 has 3 inputs (the kernel pads them to 16).
PNET_FLOPS = {"hidden": 2 * 27 * (3 * 16 + 16 * 16 + 16 * 16), "out": 2 * 27 * 16}


def run_learned(args):
    """The learned p_hat workload: exact variable-coefficient pressures of 64^3 windows (20
    samples each, 90 % train / 10 % validation), Adam training, then 128^3 inference with the
    splitting error of the learned and the linear predictors."""
    import torch

    from paper_2204_08834_gb300 import flups, learned

    nwin = args.learned_windows
    nval = max(1, nwin // 10)
    t0 = time.perf_counter()
    wins = [learned.make_window("train", w, 22)[0] for w in range(nwin)]
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    train_w, val_w = wins[:nwin - nval], wins[nwin - nval:]
    nsamp = sum(len(w.p) - 2 for w in train_w)
    steps = args.learned_epochs * nsamp
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with flups.PNet(64, 64, 64, learned.init_params()) as net:
        learned.train(net, train_w[:1], 3, lr=0.0)                 # warm-up, no change to the weights
        net.set_params(learned.init_params())
        e0.record()
        learned.train(net, train_w, steps, lr=1e-3)
        e1.record()
        torch.cuda.synchronize()
        train_ms = e0.elapsed_time(e1)
        l_net, l_lin = learned.eval_losses(net, val_w)
        params = net.params()
    del wins, train_w, val_w
    win, dt = learned.make_window("infer", 0, 6, keep_velocity=True)
    n = win.rho.shape[0]
    npts = win.rho.numel()
    ph = torch.empty_like(win.rho)
    with flups.PNet(n, n, n, params) as net, \
            flups.Plan(n, n, n, 1.0 / n, 1.0 / n, np.full(n, 1.0 / n), "periodic", "fp64",
                       torch.cuda.current_stream().cuda_stream) as plan:
        plan.set_density(win.rho)
        errs = learned.compare_predictors(net, win, dt, plan)
        reps = max(args.steps, 10)
        for _ in range(3):
            net.predict(win.rho, win.rho0, win.p[1], win.p[0], ph)
        l0 = net.launches
        e0.record()
        for _ in range(reps):
            net.predict(win.rho, win.rho0, win.p[1], win.p[0], ph)
        e1.record()
        torch.cuda.synchronize()
        pred_ms = e0.elapsed_time(e1) / reps
        launches = (net.launches - l0) / reps
        net.set_profiling(True)
        for _ in range(reps):
            net.predict(win.rho, win.rho0, win.p[1], win.p[0], ph)
        prof = {k: (ms / reps, c / reps) for k, (ms, c) in net.profile().items()}
        net.set_profiling(False)
    pk, pk_kind = peaks()
    hid_ms = prof["k_pnet_conv_hidden"][0]
    achieved = PNET_FLOPS["hidden"] * npts / (hid_ms * 1e-3) / 1e12
    mean = lambda k, i: float(np.mean([e[i] for e in errs[k]]))
    return {
        "workload": "learned p_hat: 64^3 training windows (50 droplets r U[2,6] cells, density ratio 20, "
                    "AR(1) velocity a = 0.95, smooth noise sigma 2 cells), 128^3 inference window (50 droplets "
                    "r U[4,12] cells); pressures from the exact variable-coefficient PCG solve to 1e-12",
        "samples": {"train": nsamp, "validation": nval * 20, "windows": nwin},
        "data_gen_s": round(t_data, 2),
        "train": {"steps": steps, "epochs": args.learned_epochs, "ms_per_step": round(train_ms / steps, 4),
                  "samples_per_s": round(steps / (train_ms * 1e-3), 1),
                  "mpts_per_s": round(steps * 64 ** 3 / (train_ms * 1e-3) / 1e6, 1)},
        "val_loss": {"net": round(l_net, 5), "linear": round(l_lin, 5)},
        "splitting_error_128": {"p_net": round(mean("net", 0), 5), "p_linear": round(mean("lin", 0), 5),
                                "u_net": round(mean("net", 1), 7), "u_linear": round(mean("lin", 1), 7),
                                "du_net": round(mean("net", 2), 5), "du_linear": round(mean("lin", 2), 5),
                                "steps": len(errs["net"]),
                                "definition": "e_p = |p_split - p_ex| / |p_ex|, e_u = |u_split - u_ex| / |u_ex|, "
                                              "e_du = |u_split - u_ex| / |u_ex - u**| (2-norms, mean over steps)"},
        "inference": {"grid": [n, n, n], "ms": round(pred_ms, 4), "mpts_per_s": round(npts / (pred_ms * 1e-3) / 1e6, 1),
                      "gpu_launches": launches,
                      "kernels_ms": {k: round(v[0], 4) for k, v in prof.items()}},
        "roofline": {"kernel": "k_pnet_conv_hidden (3 launches per inference)", "bound": "tensor",
                     "achieved": round(achieved, 2), "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                     "frac": round(achieved / pk["bf16_tflops"], 4), "traffic": None,
                     "algorithmic": f"{PNET_FLOPS['hidden']} flops/pt (layers 3->16, 16->16, 16->16)",
                     "peak_source": f"MEASURED_PEAKS.json bf16_tflops ({pk_kind}); tcgen05 bf16 MMA, FP32 in "
                                    "tensor memory"},
    }


def run_momentum(args):
    """The momentum predictor in front of the projection (Sec. 3.3, Eq. uss_predic) on a 512^3
    single-phase field (MAC curl of filtered noise, rms 1, nu = 1e-3, dt at CFL 0.5): the
    predictor alone in binary32-pair and binary64 arithmetic, per-kernel times from the
    library's events, and whole time steps (predictor, rhs, graph-capturable solve, correct)
    that advance the flow, all timed with CUDA events on the launch stream."""
    import torch

    from paper_2204_08834_gb300 import flups, synth

    n = 512
    h = 1.0 / n
    npts = n ** 3
    vel = synth.solenoidal_velocity(n, seed=50)
    U = max(float(np.max(np.abs(q))) for q in vel)
    nu, g = 1e-3, (0.0, 0.0, -1.0)
    dt = 0.5 * h / U
    stream = torch.cuda.current_stream().cuda_stream
    d = [torch.from_numpy(q).cuda() for q in vel]
    del vel
    o = [torch.empty_like(d[0]) for _ in range(3)]
    st = flups.momentum_state(n, n, n)
    out = {"workload": f"single-phase {n}^3 triply periodic, solenoidal u^n (MAC curl of Gaussian-filtered "
                       f"noise, sigma 4 cells, rms 1), nu = {nu}, dt = 0.5 h / max|u|, g = {g}",
           "points": npts}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, k):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    with flups.Plan(n, n, n, h, h, h, "periodic", "fp32_refine", stream) as plan:
        plan.momentum_predict(*d, *o, st, nu, g, dt, 0.0)          # first step: M^{n-1} for the AB2 calls
        for name, arith in (("pair", flups.MOM_PAIR), ("fp64", flups.MOM_FP64)):
            k = args.steps if arith == flups.MOM_PAIR else max(2, args.steps // 2)
            ms = timed(lambda: plan.momentum_predict(*d, *o, st, nu, g, dt, dt, arith), k)
            out[f"predictor_{name}"] = {"ms": round(ms, 4), "mpts_per_s": round(npts / (ms * 1e-3) / 1e6, 1),
                                        "calls": k}
        # per-kernel times of the pair path (library events)
        plan.set_profiling(True)
        for _ in range(3):
            plan.momentum_predict(*d, *o, st, nu, g, dt, dt)
        prof = {kk: (ms / 3.0, cnt / 3.0) for kk, (ms, cnt) in plan.profile().items()}
        plan.set_profiling(False)
        pk, pk_kind = peaks()
        kern = {}
        for kk, (ms, cnt) in prof.items():
            e = {"ms": round(ms, 4)}
            w = KERNEL_WORK.get(kk)
            if w and w.get("bytes"):
                gbs = w["bytes"] * npts / (ms / max(cnt, 1e-9) * 1e-3) / 1e9
                e["algorithmic_GBps"] = round(gbs, 1)
                e["hbm_frac"] = round(gbs / pk["hbm_gbs"], 4)
            kern[kk] = e
        out["kernels"] = kern
        km = kern.get("k_momentum", {})
        out["roofline"] = {"kernel": "k_momentum", "bound": "hbm", "achieved": km.get("algorithmic_GBps"),
                           "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": km.get("hbm_frac"),
                           "bytes_per_point": KERNEL_WORK["k_momentum"]["bytes"], "peak_source": pk_kind}
        # full-size accuracy of the pair path against the binary64 path (same input, Euler step)
        plan.momentum_predict(*d, *o, st, nu, g, dt, 0.0, flups.MOM_FP64)
        m64 = st.double().sum(dim=-1)
        plan.momentum_predict(*d, *o, st, nu, g, dt, 0.0, flups.MOM_PAIR)
        mp = st.double().sum(dim=-1)
        S = U * U / h + nu * U / h ** 2
        out["pair_vs_fp64_max_abs_M_over_S"] = float((mp - m64).abs().max()) / S
        del m64, mp
        # whole time steps: u^n -> u** -> projection -> u^{n+1}, the next step's u^n
        zero = torch.zeros_like(d[0])
        f = torch.empty_like(d[0])
        p = torch.empty_like(d[0])
        plan.set_density(torch.ones_like(d[0]))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        tp = tq = 0.0
        ksteps = args.steps
        rel = []
        l0 = None
        for s in range(args.warmup + ksteps):
            if s == args.warmup:
                torch.cuda.synchronize()
                l0 = plan.launches
            ev[0].record()
            plan.momentum_predict(*d, *o, st, nu, g, dt, dt if s else 0.0)
            ev[1].record()
            plan.rhs(*o, zero, zero, 0.0, 0.0, dt, f)
            plan.solve_graphable(f, p, rtol=args.rtol, max_iter=GRAPH_MAX_ITER)
            plan.correct(p, zero, zero, 0.0, 0.0, dt, *o)
            ev[2].record()
            torch.cuda.synchronize()
            if s >= args.warmup:
                tp += ev[0].elapsed_time(ev[1])
                tq += ev[1].elapsed_time(ev[2])
                rel.append(plan.solve_result(rtol=args.rtol).rel_res)
            d, o = o, d
        launches = plan.launches - l0
    ms = (tp + tq) / ksteps
    out["time_step"] = {"ms": round(ms, 4), "mpts_per_s": round(npts / (ms * 1e-3) / 1e6, 1),
                        "predictor_ms": round(tp / ksteps, 4), "projection_ms": round(tq / ksteps, 4),
                        "steps": ksteps, "max_rel_res": max(rel), "gpu_launches_per_step": launches / ksteps,
                        "step": "momentum_predict (pair, AB2) + rhs + solve_graphable (FP32+refine, "
                                f"rtol {args.rtol:g}) + correct; u^(n+1) feeds the next step"}
    del d, o, st
    torch.cuda.empty_cache()
    return out


def run_vof(args):
    """The VoF step (Sec. 3.1, App. A: MTHINC reconstruction, split advection x, y, z, the
    divergence correction) on a 256^3 periodic box of 30 droplets (r U[4,12] cells, tanh
    profile 1.5 cells wide) in the solenoidal single-phase velocity of the momentum leg, CFL
    0.5, beta_th = 2; time per step with CUDA events, per-kernel times from the library's events,
    and the change of sum(phi) over the timed steps."""
    import torch

    from paper_2204_08834_gb300 import flups, synth

    n = 256
    h = 1.0 / n
    rng = np.random.default_rng(70)
    x = np.arange(n) + 0.5
    phi = np.zeros((n, n, n))
    for _ in range(30):
        c = rng.uniform(0, n, 3)
        rad = rng.uniform(4.0, 12.0)
        dd = [np.minimum(np.abs(x - c[a]), n - np.abs(x - c[a])) for a in range(3)]
        r = np.sqrt(dd[0][None, None, :] ** 2 + dd[1][None, :, None] ** 2 + dd[2][:, None, None] ** 2)
        phi = np.maximum(phi, 0.5 * (1.0 - np.tanh((r - rad) / 0.75)))
    vel = synth.solenoidal_velocity(n, seed=71)
    U = max(float(np.max(np.abs(q))) for q in vel)
    dt = 0.5 * h / U
    d = torch.from_numpy(phi).cuda()
    v = [torch.from_numpy(q).cuda() for q in vel]
    del phi, vel
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with flups.Plan(n, n, n, h, h, np.full(n, h), "periodic", "fp32_refine", torch.cuda.current_stream().cuda_stream) \
            as plan:
        for _ in range(args.warmup):
            plan.vof_step(d, *v, dt, 2.0)
        torch.cuda.synchronize()
        m0 = float(d.sum())
        k = args.steps
        e0.record()
        for _ in range(k):
            plan.vof_step(d, *v, dt, 2.0)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        m1 = float(d.sum())
        status = plan.sync(check=False)
        plan.set_profiling(True)
        plan.vof_step(d, *v, dt, 2.0)
        prof = plan.profile()
        plan.set_profiling(False)
        lo, hi = float(d.min()), float(d.max())
    pk, pk_kind = peaks()
    kern = {}
    for kk, (kms, cnt) in prof.items():
        e = {"ms": round(kms, 4), "launches": cnt}
        w = KERNEL_WORK.get(kk)
        if w and w.get("bytes") and cnt:
            per = 3 if kk != "k_vof_update" else 4
            gbs = w["bytes"] * n ** 3 * per / (kms * 1e-3) / 1e9
            e["algorithmic_GBps"] = round(gbs, 1)
            e["hbm_frac"] = round(gbs / pk["hbm_gbs"], 4)
        kern[kk] = e
    return {"workload": "VoF step, 256^3 periodic, 30 droplets r U[4,12] cells (tanh profile 1.5 cells), "
                        "solenoidal velocity (MAC curl of filtered noise), CFL 0.5, beta_th = 2",
            "ms_per_step": round(ms, 4), "mcells_per_s": round(n ** 3 / (ms * 1e-3) / 1e6, 1), "steps": k,
            "mass_rel_change": (m1 - m0) / m0, "phi_range": [lo, hi], "status": flups.status_string(status),
            "kernels": kern,
            "arithmetic": "reconstruction and fluxes FP32 (d_th by Newton on the volume equation), updates FP64"}


def run_ends(args):
    """The Poisson solve in the generality of Sec. 3.3.1: a closed box with homogeneous Neumann
    ends in x and y (cosine series along x and y) and walls in z with tanh-stretched spacing
    (beta 1.5), 512 x 512 x 256 (the two-layer Rayleigh-Benard shape in a closed cell), f ~ N(0,1)
    seeded; FP32 transforms + FP64 defect correction to rtol vs the FP64 direct solve, CUDA
    events around whole solves on the launch stream."""
    import torch

    from paper_2204_08834_gb300 import flups, synth

    nx, ny, nz = 512, 512, 256
    dzf = synth.stretched_dzf(nz, 1.0, 1.5)
    dx = dy = 2.0 / nx
    npts = nx * ny * nz
    stream = torch.cuda.current_stream().cuda_stream
    f = torch.from_numpy(np.random.default_rng(60).standard_normal((nz, ny, nx))).cuda()
    p = torch.empty_like(f)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": "closed box 512x512x256: Neumann ends in x and y (cosine series), z walls with "
                       "tanh-stretched dz (beta 1.5), dx = dy = 2/512, f ~ N(0,1) seeded", "points": npts}
    pk, pk_kind = peaks()
    for prec in ("fp32_refine", "fp64"):
        rtol = args.rtol if prec == "fp32_refine" else 0.0
        k = args.steps if prec == "fp32_refine" else max(2, args.steps // 2)
        with flups.Plan(nx, ny, nz, dx, dy, dzf, "walls", prec, stream, bcx="neumann", bcy="neumann") as plan:
            for _ in range(args.warmup):
                info = plan.solve(f, p, rtol=rtol, max_iter=12)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(k):
                info = plan.solve(f, p, rtol=rtol, max_iter=12)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / k
            entry = {"ms_per_solve": round(ms, 4), "mpts_per_s": round(npts / (ms * 1e-3) / 1e6, 1), "solves": k,
                     "iters": info.iters, "rel_res": info.rel_res}
            if prec == "fp32_refine":
                plan.set_profiling(True)
                plan.solve(f, p, rtol=rtol, max_iter=12)
                prof = plan.profile()
                plan.set_profiling(False)
                kern = {}
                for kk, (kms, cnt) in sorted(prof.items(), key=lambda kv: -kv[1][0]):
                    e = {"ms": round(kms, 4), "regions": cnt}
                    w = KERNEL_WORK.get(kk)
                    if kk == "k_res_ends" and cnt:
                        gbs = w["bytes"] * npts / (kms / cnt * 1e-3) / 1e9
                        e["algorithmic_GBps"] = round(gbs, 1)
                        e["hbm_frac"] = round(gbs / pk["hbm_gbs"], 4)
                    kern[kk] = e
                entry["kernels"] = kern
            out[prec] = entry
    del f, p
    torch.cuda.empty_cache()
    return out


def cpu_baseline(c, f, p32, p64):
    """The FP64 oracle (numpy, as it stands) on the host cores: one direct solve of the bench
    workload's own right-hand side f (the step's f, copied from the GPU) single-threaded, and
    the same solve with its transforms on every host core (scipy.fft workers); plus the error
    of the GPU's p against that solution."""
    import oracle

    nz, ny, nx = c.shape
    g = oracle.make_grid(nx, ny, nz, c.dx, c.dy, c.dzf, c.bc)
    t0 = time.perf_counter()
    po = oracle.solve(f, g)
    t1 = time.perf_counter()
    ncores = os.cpu_count() or 1
    oracle.solve(f, g, workers=ncores)
    t2 = time.perf_counter()
    hi = host_info()
    return {"value": round(c.npts / (t1 - t0) / 1e6, 3), "unit": "Mpts/s", "cores": 1, "kind": "oracle",
            "sample": f"one FP64 direct solve (oracle.solve) of the {nx}x{ny}x{nz} bench right-hand side, "
                      "numpy single-threaded",
            "nproc": hi["nproc"], "cpu_model": hi["cpu_model"],
            "threaded": {"value": round(c.npts / (t2 - t1) / 1e6, 3), "unit": "Mpts/s", "cores": ncores,
                         "kind": "oracle, transforms on all host cores (scipy.fft workers)"},
            "error_vs_oracle": {"fp32_refine": rel_err(p32, po), "fp64": rel_err(p64, po),
                                "definition": "|p - p_oracle|_2 / |p_oracle|_2 of the GPU solves of the same f"}}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle's direct solve timed on the host cores (no reference
    program exists); each step solves the 256^3 emulsion right-hand side, a bounded sample of
    the 512^3 emulsion workload (one 512^3 oracle solve takes tens of seconds)."""
    if rank != 0:
        return 0
    import oracle
    from paper_2204_08834_gb300 import synth

    c = synth.emulsion(256, ratio=10.0)
    g = oracle.make_grid(256, 256, 256, c.dx, c.dy, c.dzf, c.bc)
    f = oracle.rhs(c.u, c.v, c.w, c.rho, c.pn, c.pnm1, 2.0, 1.0, c.dt, g)
    tot = 0.0
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.solve(f, g)
        t1 = time.perf_counter()
        if s >= args.warmup:
            tot += t1 - t0
    val = args.steps * c.npts / tot / 1e6
    hi = host_info()
    line = {
        "impl": "reference", "metric": METRIC, "value": round(val, 3), "unit": "Mpts/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * tot / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "emulsion 256^3 triply periodic, 200 droplets, density ratio 10 (bounded sample "
                               "of the 512^3 emulsion workload)",
                   "step": "oracle.solve: FP64 direct eigen-expansion solve of the step's right-hand side",
                   "threads": 1},
        "cpu_baseline": {"value": round(val, 3), "unit": "Mpts/s", "cores": 1, "kind": "oracle",
                         "sample": "one 256^3 emulsion solve per step", "nproc": hi["nproc"],
                         "cpu_model": hi["cpu_model"]},
        "e2e": {"value": round(val, 3), "unit": "Mpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="emulsion512", choices=list(WORKLOADS))
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-cufft", action="store_true")
    ap.add_argument("--no-momentum", action="store_true")
    ap.add_argument("--no-ends", action="store_true")
    ap.add_argument("--no-vof", action="store_true")
    ap.add_argument("--configs", default="emulsion256,emulsion512_r1,two_layer512,two_layer1024",
                    help="comma-separated further workloads timed with both precisions (empty: none)")
    ap.add_argument("--learned-windows", type=int, default=100,
                    help="64^3 training windows of 20 samples (default 100: 2000 samples)")
    ap.add_argument("--learned-epochs", type=int, default=3)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    if world > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}))
        return 1

    out = run_ours(args, rank, world, local)
    if world > 1:
        torch.distributed.barrier()
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    c, npts, m = out["c"], out["npts"], out["m"]
    r = rates(m, world)
    k32 = r["fp32_refine"]["steps"]
    ms_solve = r["fp32_refine"]["solve_ms"]
    ms_step = r["fp32_refine"]["projection_ms"]
    value = r["fp32_refine"]["solve_mpts"]
    pk, pk_kind = peaks()
    prof = out["prof"]
    tot_prof = sum(ms for ms, n in prof.values()) or 1.0

    # solves in the profiled steps: the first forward x pass runs once per solve
    nsolve = max(prof.get("k_xfwd_f32", (0.0, 1.0))[1], 1e-9)
    p32 = p32_first(c)

    def kbytes(k, n):
        w = KERNEL_WORK.get(k)
        if not w or not w.get("bytes"):
            return None
        return solve_bytes_per_point(k, n / nsolve, p32) if k in SOLVE_KERNELS else w["bytes"]

    def kernel_entry(k, ms, n):
        e = {"ms_per_step": round(ms, 4), "launch_regions_per_step": n, "share": round(ms / tot_prof, 4)}
        b = kbytes(k, n)
        if b and n:
            gbs = b * npts / (ms / n * 1e-3) / 1e9
            e["algorithmic_GBps"] = round(gbs, 1)
            e["hbm_frac"] = round(gbs / pk["hbm_gbs"], 4)
            e["bytes_per_point"] = round(b, 2)
        return e

    kernels = {k: kernel_entry(k, ms, n) for k, (ms, n) in sorted(prof.items(), key=lambda kv: -kv[1][0])}
    solve_prof = {k: v for k, v in prof.items() if k in SOLVE_KERNELS}
    dom = max(solve_prof, key=lambda k: solve_prof[k][0])
    work = dict(KERNEL_WORK.get(dom, {"bound": "hbm", "bytes": None}))
    if work.get("bytes"):
        work["bytes"] = round(kbytes(dom, prof[dom][1]), 2)
    dom_ms_per_region = prof[dom][0] / max(prof[dom][1], 1e-9)
    achieved = (work["bytes"] or 0) * npts / (dom_ms_per_region * 1e-3) / 1e9
    peak, unit, psrc = pk["hbm_gbs"], "GB/s", f"MEASURED_PEAKS.json hbm_gbs ({pk_kind})"
    # the solve as a whole against its compulsory traffic (bytes per point of the passes it ran)
    solve_bytes = sum(kbytes(k, n) * n for k, (ms, n) in solve_prof.items() if kbytes(k, n)) / nsolve
    solve_ms_prof = sum(ms for ms, n in solve_prof.values()) / nsolve
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "Mpts/s",
        "n_gpus": world,
        "steps": k32,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64+f32",
        "data": "synthetic",
        "config": {
            "workload": WORKLOADS[args.workload]["desc"] + "; FP32 transforms + FP64 residual refinement to "
                        f"rel. residual {args.rtol:g}",
            "grid": list(c.shape[::-1]),
            "step": "set_density + rhs + solve + correct (one projection)",
            "value": "grid points / CUDA-event time of the solve call (f -> p at the residual) inside each step; "
                     "the whole step's rate is projection_mpts",
            "l2": "inputs larger than L2 (each field 1 GiB at 512^3)",
            "timing": "sum of per-step CUDA-event intervals on the launch stream; the copy that restores u** "
                      "between steps is outside the events",
            "solve_form": f"flups_solve_graphable (at most {GRAPH_MAX_ITER} FP32 solves, device-side exit at rtol); "
                          "rel_res read after each step",
            "parallelism": f"replicas x{world}",
        },
        "solve_ms": ms_solve,
        "projection_mpts": r["fp32_refine"]["projection_mpts"],
        "breakdown_ms": r["fp32_refine"]["breakdown_ms"],
        "iters": r["fp32_refine"]["iters"],
        "rel_res": r["fp32_refine"]["rel_res"],
        "fp64": {"solve_mpts": r["fp64"]["solve_mpts"], "solve_ms": r["fp64"]["solve_ms"],
                 "projection_mpts": r["fp64"]["projection_mpts"], "breakdown_ms": r["fp64"]["breakdown_ms"],
                 "steps": r["fp64"]["steps"], "rel_res": r["fp64"]["rel_res"],
                 "solve": "FP64 direct eigen-expansion solve (no residual evaluation in the timed region)"},
        "speedup_fp32_refine_vs_fp64": round(value / r["fp64"]["solve_mpts"], 3),
        "roofline": {
            "kernel": dom,
            "bound": work["bound"],
            "achieved": round(achieved, 4),
            "peak": peak,
            "unit": unit,
            "frac": round(achieved / peak, 4),
            "traffic": MEASURED_TRAFFIC_PER_LAUNCH.get((args.workload, dom)),
            "traffic_note": ("bytes per launch: ncu DRAM read + write (dram__bytes_read.sum + "
                             "dram__bytes_write.sum), see MEASURED_TRAFFIC_PER_LAUNCH"
                             if (args.workload, dom) in MEASURED_TRAFFIC_PER_LAUNCH else None),
            "per_launch_ms": round(dom_ms_per_region, 4),
            "peak_source": psrc,
            "algorithmic": {k: v for k, v in work.items() if k != "bound"},
            "scope": "the kernel that takes most of the FP32+refine solve's time (library CUDA events)",
            "solve": {"bytes_per_point": round(solve_bytes, 2),
                      "achieved": round(solve_bytes * npts / (solve_ms_prof * 1e-3) / 1e9, 1),
                      "frac": round(solve_bytes * npts / (solve_ms_prof * 1e-3) / 1e9 / peak, 4),
                      "ms": round(solve_ms_prof, 4),
                      "note": "the whole solve: compulsory bytes per point of every pass it ran over the "
                              "kernels' summed event time"},
        },
        "kernels": kernels,
        "gpu_launches": int(m["fp32_refine"]["launches"]),
        "clocks": out["clocks"],
    }
    wc = KERNEL_WORK["k_correct"]
    if "k_correct" in prof:
        cms = prof["k_correct"][0] / max(prof["k_correct"][1], 1e-9)
        floor_ms = wc["fp64_instr"] * npts / (FP64_TFLOPS_MEASURED / 2.0 * 1e12) * 1e3
        kernels["k_correct"]["fp64_pipe"] = {"instr_per_point": wc["fp64_instr"], "floor_ms": round(floor_ms, 4),
                                             "frac": round(floor_ms / cms, 4),
                                             "rate": "FP64 pipe instructions at the DFMA rate measured by "
                                                     "microbench/peaks.cu"}
        kernels["k_correct"]["measured_traffic_per_launch"] = MEASURED_TRAFFIC_PER_LAUNCH.get(
            (args.workload, "k_correct"))
    if "e2e" in out:
        t_e2e, ne, e2e_rel = out["e2e"]
        line["e2e"] = {"value": round(world * npts * ne / t_e2e / 1e6, 2), "unit": "Mpts/s",
                       "h2d_bytes_per_step": 8 * npts, "d2h_bytes_per_step": 8 * npts,
                       "steps": ne, "rel_res": e2e_rel,
                       "call": "flups_solve_host (FP32+refine to rtol; f in, p out through pinned host buffers)"}
    if out.get("cufft"):
        cu = out["cufft"]
        cu["ours_fp64_solve_mpts"] = line["fp64"]["solve_mpts"]
        cu["ours_fp32_refine_solve_mpts"] = value
        line["cufft_baseline"] = cu
    for key in ("ensemble", "learned", "momentum", "ends", "vof"):
        if key in out:
            line[key] = out[key]
    if out["configs"]:
        line["configs"] = out["configs"]
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(c, m["f"], m["fp32_refine"]["p"], m["fp64"]["p"])
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
