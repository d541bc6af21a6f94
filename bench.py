"""Benchmark of the SIPG viscous operator apply (and the solver around it) on GB300.

Workload (the throughput configuration): unit cube, 32^3 affine hexahedra,
velocity degree k = 3 (6,291,456 DoFs), Carreau-Yasuda viscosity (eta0 = 1,
eta_inf = 1e-3, lambda = 1, a = 2, b = 0.5) evaluated from the gradient of a
seeded divergence-free Fourier velocity (8 modes); one step = one FP64-accurate apply
y = A_visc(nu) x through the C ABI (float-float arithmetic on the FP32 pipe by
default, ``--arith f64`` for native FP64; both match the FP64 oracle to 1e-12). Inputs exceed L2: four rotating x/y vector
pairs (403 MB) plus the stored viscosity (42 MB).

Prints ONE JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle
(explicit element matrices) on a bounded sample of the same workload instead.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CELLS, K_U = 32, 3
METRIC = "GDoF/s of SIPG viscous op apply"
WORKLOAD = "box 32^3 affine hexes, k=3 velocity (6,291,456 DoFs), Carreau-Yasuda nu from Fourier field"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--no-extras", action="store_true", help="skip the extra solve / precision lines")
    p.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing (profiling runs)")
    p.add_argument("--arith", default="f64ff", choices=["f64", "f64ff"],
                   help="arithmetic of the timed apply: native FP64 or float-float (FP64-accurate)")
    p.add_argument("--channel-steps", type=int, default=10, help="timed steps of the channel extras")
    p.add_argument("--setup-lag", type=int, default=1, help="mg_setup_lag of the channel extras")
    p.add_argument("--extra", default=None,
                   choices=["mass", "picard", "step", "trilinear", "channel", "jchannel", "f32apply", "serve"],
                   help="run one extra workload alone and print its JSON (profiling runs)")
    return p.parse_args()


def run_extra(name, steps=10, lag=1):
    """One extra workload on its own (the commands of the ncu summaries in profiles/)."""
    import torch

    from paper_2506_14424_gb300 import Context, inputs
    torch.cuda.set_device(0)
    if name == "step":
        out = step_extras()
    elif name == "trilinear":
        out = trilinear_extras()
    elif name == "channel":
        out = channel_extras(steps=steps, setup_lag=lag)
    elif name == "jchannel":
        out = channel_extras(steps=steps, jitter=True, setup_lag=lag)
    elif name == "f32apply":
        out = f32_apply_extra()
    elif name == "serve":
        out = serving_full()
    else:
        ctx = Context(N_CELLS, N_CELLS, N_CELLS, K_U, krylov_arith="f64ff")
        n = ctx.n_dofs("viscous")
        if name == "mass":
            xs = [torch.tensor(inputs.uniform_vector(n, seed=100 + i), device="cuda") for i in range(4)]
            ys = [torch.empty_like(xs[0]) for _ in range(4)]
            out = mass_timings(ctx, xs, ys, torch.cuda.current_stream())
        else:
            out = picard_extras(ctx)
        ctx.close()
    print(json.dumps({"extra": name, "result": out}), flush=True)


def f32_apply_extra(reps=40):
    """FP32 viscous apply (the multigrid level operator) on the 32^3, k = 3 workload,
    rotating four vector pairs larger than L2 together."""
    import torch

    from paper_2506_14424_gb300 import Context, inputs
    ctx = Context(N_CELLS, N_CELLS, N_CELLS, K_U)
    n = ctx.n_dofs("viscous")
    u = torch.tensor(fourier_velocity(ctx.node_points("viscous", 0)), device="cuda")
    ctx.set_viscosity(inputs.carreau_blood_like(), u)
    xs = [torch.tensor(inputs.uniform_vector(n, seed=100 + i), device="cuda", dtype=torch.float32) for i in range(4)]
    ys = [torch.empty_like(xs[0]) for _ in range(4)]
    ms = time_apply(ctx, "viscous", xs[0], ys[0], reps, torch.cuda.current_stream(), rotate=(xs, ys))
    ctx.close()
    return {"ms": ms, "gdofs": n / ms / 1e6, "n_dofs": n}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ----------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        # the raw samples (the summary goes into the JSON line); SIPG_BENCH_DIR keeps them
        out_dir = os.environ.get("SIPG_BENCH_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ shared input
def fourier_velocity(node_points):
    from paper_2506_14424_gb300 import inputs
    modes = inputs.fourier_modes(1)
    C = N_CELLS ** 3
    u = inputs.fourier_field(node_points.reshape(-1, 3), modes)
    return u.reshape(C, -1, 3).transpose(0, 2, 1).reshape(-1)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except Exception:
        return {}


def traffic_record(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if still valid."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(p)).get(kernel_key)
    except Exception:
        return None
    if not rec:
        return None
    src = open(os.path.join(ROOT, "paper_2506_14424_gb300", "csrc", rec["source"]), "rb").read()
    if hashlib.sha256(src).hexdigest()[:16] != rec["source_sha"]:
        return None
    return rec["dram_bytes_per_launch"]


# ALU peaks of the GPU, measured at start-up by the library's FMA-chain kernel
# (sipg_alu_peak): FP64 and FP32 TFLOP/s. The FP64-equivalent peak of float-float
# arithmetic on the FP32 pipe is the FP32 multiply-add rate over 12 instructions per
# float-float multiply-add (exact product 4, TwoSum 6, low-word adds 2), 2 flops each.
FF_INSTR_PER_MA = 12
_PEAKS = {}


def alu_peaks():
    """{'f64': TFLOP/s, 'f32': TFLOP/s, 'f64ff': TFLOP/s}, measured once per process."""
    if not _PEAKS:
        from paper_2506_14424_gb300 import alu_peak
        f64 = max(alu_peak("f64") for _ in range(3))
        f32 = max(alu_peak("f32") for _ in range(3))
        _PEAKS.update({"f64": f64, "f32": f32, "f64ff": f32 / FF_INSTR_PER_MA})
    return _PEAKS


# Algorithmic flops per DoF of the k=3 viscous apply (minimal sum-factorised count).
FLOP_PER_DOF = 250.0


def algorithmic_bytes(n_dofs, cells, n):
    return 16.0 * n_dofs + 8.0 * (cells * n ** 3 + 6 * cells * n ** 2)


def max_over_ranks(value, world, device="cpu"):
    """Largest value over the ranks of the default process group (the bench
    times every rank and reports the slowest)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def aggregate_throughput(units_per_rank, ms_max, world):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / (ms_max * 1e-3)


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2506_14424_gb300 import Context, inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    ctx = Context(N_CELLS, N_CELLS, N_CELLS, K_U, krylov_arith=args.arith)  # e2e uses the same arithmetic
    n = ctx.n_dofs("viscous")
    u = torch.tensor(fourier_velocity(ctx.node_points("viscous", 0)), device="cuda")
    ctx.set_viscosity(inputs.carreau_blood_like(), u)
    del u
    pairs = 4
    xs = [torch.tensor(inputs.uniform_vector(n, seed=100 + i), device="cuda") for i in range(pairs)]
    ys = [torch.empty_like(xs[0]) for _ in range(pairs)]
    for i in range(args.warmup):
        ctx.apply("viscous", xs[i % pairs], ys[i % pairs], arith=args.arith)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(args.steps):
        ctx.apply("viscous", xs[i % pairs], ys[i % pairs], arith=args.arith)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, device="cuda")
    if world > 1:
        dist.barrier()
    ms_step = ms / args.steps
    value = aggregate_throughput(n * args.steps, ms, world) / 1e9

    # end to end through the C ABI with pinned host buffers (copies inside the region)
    xh_t = torch.empty(n, dtype=torch.float64, pin_memory=True)
    yh_t = torch.empty(n, dtype=torch.float64, pin_memory=True)
    xh, yh = xh_t.numpy(), yh_t.numpy()
    xh[:] = inputs.uniform_vector(n, seed=200)
    for _ in range(2):
        ctx.apply_host("viscous", xh, out=yh)
    t0 = time.perf_counter()
    e2e_steps = max(3, min(args.steps, 20))
    for _ in range(e2e_steps):
        ctx.apply_host("viscous", xh, out=yh)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": n / e2e_s / 1e9, "unit": "GDoF/s", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n}

    C = N_CELLS ** 3
    nb = K_U + 1
    alg_bytes = algorithmic_bytes(n, C, nb)
    pk = alu_peaks()
    key = "apply_kernel<4,3,double>" if args.arith == "f64" else "apply_kernel<4,3,ff>"
    roof = roofline(ms_step, n, alg_bytes, args.arith, pk, key)
    # the binary64 kernel on the same inputs, as its own field
    ms64 = time_apply(ctx, "viscous", xs[0], ys[0], max(10, min(args.steps, 50)), stream, arith="f64",
                      rotate=(xs, ys))
    binary64 = {"value": n / ms64 / 1e6, "unit": "GDoF/s", "ms_per_apply": ms64, "dtype": "f64",
                "roofline": roofline(ms64, n, alg_bytes, "f64", pk, "apply_kernel<4,3,double>")}
    extras = {}
    if not args.no_extras and rank == 0:
        extras = gpu_extras(ctx, xs, ys, stream)
    line = {"metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.arith == "f64" else "f32x2 (float-float, FP64-accurate)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": [N_CELLS] * 3, "k_u": K_U, "n_dofs": n, "arith": args.arith,
                       "l2": "inputs larger than L2: 4 rotating x/y pairs (403 MB) + 42 MB stored nu",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "clocks": clk, "e2e": e2e, "gpu_launches": args.steps * (2 if args.arith == "f64ff" else 1),
            "roofline": roof, "binary64": binary64,
            "alu_peaks_tflops": {k: round(v, 3) for k, v in pk.items()}}
    if rank == 0:
        line["cpu_baseline"] = None if args.no_cpu_baseline else cpu_baseline(sample_cells=1024)
        if line["cpu_baseline"]:
            line["cpu_baseline"]["note"] = ("the explicit-block Python oracle (element blocks rebuilt per cell), "
                                            "not a tuned CPU implementation: a correctness reference, not a "
                                            "speed baseline")
        line["extras"] = extras
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def roofline(ms, n, alg_bytes, arith, pk, key):
    """ALU roofline of one viscous apply (the bound of these kernels) with the HBM fraction beside it."""
    flops = FLOP_PER_DOF * n
    achieved = flops / (ms * 1e-3) / 1e12
    peak = pk[arith]
    hbm = peaks().get("hbm_gbs", 6686.1)
    src = {"f64": "measured FP64 FMA rate (sipg_alu_peak)", "f32": "measured FP32 FMA rate (sipg_alu_peak)",
           "f64ff": "FP64-equivalent float-float peak: measured FP32 FMA rate / 12 instructions per "
                    "float-float multiply-add"}[arith]
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic_record(key), "kernel": key, "peak_source": src,
            "hbm_achieved_gbs": alg_bytes / (ms * 1e-3) / 1e9, "hbm_peak_gbs": hbm,
            "hbm_frac": alg_bytes / (ms * 1e-3) / 1e9 / hbm,
            "algorithmic_bytes_per_launch": alg_bytes, "algorithmic_flops_per_launch": flops}


def time_apply(ctx, op, x, y, reps, stream, warm=3, arith=None, rotate=None):
    """CUDA-event time of one apply (ms); rotate=(xs, ys) cycles through vectors larger than L2."""
    import torch
    X, Y = rotate if rotate else ([x], [y])
    for i in range(warm):
        ctx.apply(op, X[i % len(X)], Y[i % len(Y)], arith=arith)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(reps):
        ctx.apply(op, X[i % len(X)], Y[i % len(Y)], arith=arith)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def gpu_extras(ctx, xs, ys, stream):
    import numpy as np
    import torch

    from paper_2506_14424_gb300 import Context, inputs

    out = {}
    n = ctx.n_dofs("viscous")
    yref = ctx.apply("viscous", xs[0])
    pk = alu_peaks()
    for arith in ("f64", "f64ff"):
        ms = time_apply(ctx, "viscous", xs[0], ys[0], 20, stream, arith=arith, rotate=(xs, ys))
        ctx.apply("viscous", xs[0], ys[0], arith=arith)
        diff = ((ys[0] - yref).abs().max() / yref.abs().max()).item()
        tf = FLOP_PER_DOF * n / (ms * 1e-3) / 1e12
        out[f"viscous_{arith}_apply"] = {"ms": ms, "gdofs": n / ms / 1e6, "rel_diff_vs_f64": diff,
                                         "alu_frac": tf / pk[arith], "alu_peak_tflops": pk[arith]}
    # FP32 multigrid-level apply (the V-cycle's operator), rotating vectors larger than L2
    x32 = [x.float() for x in xs]
    y32 = [y.float() for y in ys]
    ms = time_apply(ctx, "viscous", x32[0], y32[0], 40, stream, rotate=(x32, y32))
    ctx.apply("viscous", x32[0], y32[0])
    d32 = ((y32[0].double() - yref).abs().max() / yref.abs().max()).item()
    tf = FLOP_PER_DOF * n / (ms * 1e-3) / 1e12
    out["viscous_f32_apply"] = {"ms": ms, "gdofs": n / ms / 1e6, "rel_diff_vs_f64": d32,
                                "alu_frac": tf / pk["f32"], "alu_peak_tflops": pk["f32"],
                                "hbm_frac": 12.0 * n / (ms * 1e-3) / 1e9 / peaks().get("hbm_gbs", 6686.1),
                                "kernel": "apply_tpc_kernel<4,3> (register-tiled)"}
    del x32, y32
    npr = ctx.n_dofs("poisson")
    xp = torch.tensor(inputs.uniform_vector(npr, seed=300), device="cuda")
    yp = torch.empty_like(xp)
    ms = time_apply(ctx, "poisson", xp, yp, 50, stream)
    out["poisson_f64_apply_k2"] = {"ms": ms, "gdofs": npr / ms / 1e6, "n_dofs": npr}
    ms = time_apply(ctx, "poisson", xp, yp, 50, stream, arith="f64ff")
    out["poisson_f64ff_apply_k2"] = {"ms": ms, "gdofs": npr / ms / 1e6, "n_dofs": npr,
                                     "l2": "warm: x, y (14 MB) stay in L2"}
    # L2-cold: 24 rotating pairs (340 MB) so that every apply reads x from HBM
    xps = [torch.tensor(inputs.uniform_vector(npr, seed=400 + i), device="cuda") for i in range(24)]
    yps = [torch.empty_like(xps[0]) for _ in xps]
    for arith in ("f64", "f64ff"):
        ms = time_apply(ctx, "poisson", xps[0], yps[0], 48, stream, arith=arith, rotate=(xps, yps))
        out[f"poisson_{arith}_apply_k2_l2cold"] = {"ms": ms, "gdofs": npr / ms / 1e6, "n_dofs": npr,
                                                   "l2": "cold: 24 rotating x/y pairs (340 MB)"}
    del xps, yps
    # the small FP64 configuration: 4^3 cells, k = 2, analytic viscosity, Jacobi-preconditioned
    # CG to 1e-8 against the manufactured load (5,184 DoFs)
    c1 = Context(4, 4, 4, 2, mg_precision="f64")
    c1.set_viscosity({"law": "analytic"})
    b1 = c1.rhs_manufactured("velocity")
    c1.solve("viscous", b1, rtol=1e-8, precond="jacobi", maxit=2000, check=False)
    torch.cuda.synchronize()
    x1, st1 = c1.solve("viscous", b1, rtol=1e-8, precond="jacobi", maxit=2000, check=False)
    out["jacobi_cg_4cubed_k2"] = {"seconds": st1["seconds"], "iterations": st1["iterations"],
                                  "rel_residual": st1["rel_residual"], "status": st1["status"],
                                  "n_dofs": c1.n_dofs(), "solves_per_s": 1.0 / st1["seconds"]}
    c1.close()
    # mixed-precision vs all-FP64 multigrid solve, 16^3 cells, k = 4, sinker viscosity
    solves = []
    sink = inputs.sinker(seed=2, count=8, radius=0.1, nu_max=1.0)
    for contrast in (1.0, 1e2, 1e4, 1e6):
        sink["nu_max"] = contrast
        row = {"contrast": contrast}
        for prec in ("f32", "f64"):  # the DG hierarchy (every level discontinuous)
            c3 = Context(16, 16, 16, 4, mg_precision=prec, mg_cph=False)
            c3.set_viscosity(sink)
            nn = c3.n_dofs("viscous")
            ustar = torch.tensor(inputs.uniform_vector(nn, seed=3), device="cuda")
            b = c3.apply("viscous", ustar)
            _, st = c3.solve("viscous", b, rtol=1e-8, precond="mg", maxit=1000, check=False)
            x, st = c3.solve("viscous", b, rtol=1e-8, precond="mg", maxit=1000, check=False)
            err = (torch.linalg.norm(x - ustar) / torch.linalg.norm(ustar)).item()
            row["dg_" + prec] = {"seconds": st["seconds"], "iterations": st["iterations"],
                                 "rel_residual": st["rel_residual"], "status": st["status"],
                                 "rel_error_vs_ustar": err}
            c3.close()
        row["mixed_speedup"] = row["dg_f64"]["seconds"] / row["dg_f32"]["seconds"]
        # the default on a box: the cph hierarchy (continuous levels below the DG level),
        # FP32 V-cycle
        c3 = Context(16, 16, 16, 4, mg_precision="f32")
        c3.set_viscosity(sink)
        nn = c3.n_dofs("viscous")
        ustar = torch.tensor(inputs.uniform_vector(nn, seed=3), device="cuda")
        b = c3.apply("viscous", ustar)
        c3.solve("viscous", b, rtol=1e-8, precond="mg", maxit=1000, check=False)
        x, st = c3.solve("viscous", b, rtol=1e-8, precond="mg", maxit=1000, check=False)
        row["cph_f32_default"] = {"seconds": st["seconds"], "iterations": st["iterations"],
                                  "rel_residual": st["rel_residual"], "status": st["status"],
                                  "rel_error_vs_ustar": (torch.linalg.norm(x - ustar) / torch.linalg.norm(ustar)).item()}
        c3.close()
        solves.append(row)
    out["sinker_mg_solves_16cubed_k4"] = solves
    # each further workload on its own: a failure is recorded in its entry, the line still prints
    for key, fn in (("mass_32cubed_k3", lambda: mass_timings(ctx, xs, ys, stream)),
                    ("picard_viscous_step_32cubed_k3", lambda: picard_extras(ctx)),
                    ("splitting_step_32cubed_k3", step_extras),
                    ("trilinear_cells_32cubed_k3", trilinear_extras),
                    ("bfs_channel_steps", channel_extras),
                    ("bfs_jittered_channel_steps", lambda: channel_extras(jitter=True, steps=3)),
                    ("components_16cubed_k4", lambda: component_timings(stream)),
                    ("serving", serving_extras)):
        try:
            out[key] = fn()
        except Exception as exc:  # noqa: BLE001 - reported in the JSON line
            out[key] = {"error": f"{type(exc).__name__}: {exc}"}
    return out


def mass_timings(ctx, xs, ys, stream, reps=40):
    """Cell mass matrix and its inverse on the bench mesh: HBM-bound streaming
    kernels (16 bytes per DoF), rotating over the bench's x/y pairs (> L2)."""
    import torch
    n = ctx.n_dofs("viscous")
    hbm = peaks().get("hbm_gbs", 6686.1)
    out = {}
    for arith in ("f64", "f64ff"):
        for inverse in (False, True):
            def run(i):
                ctx.mass("viscous", xs[i % len(xs)], ys[i % len(ys)], coeff=2.0, arith=arith, inverse=inverse)
            for i in range(3):
                run(i)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(reps):
                run(i)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            gbs = 16.0 * n / (ms * 1e-3) / 1e9
            out[f"{'inverse_' if inverse else ''}mass_{arith}"] = {"ms": ms, "gbs": gbs, "hbm_frac": gbs / hbm}
    return out


def picard_extras(ctx, dt=1e-2):
    """Viscous step of BDF2 (gamma_0 = 3/2) with the Carreau-Yasuda law treated
    implicitly: Picard updates with and without Aitken relaxation, each linear
    solve to 1e-3 of its initial residual, nonlinear tolerance 1e-6."""
    import numpy as np
    import torch

    from paper_2506_14424_gb300 import inputs
    k = ctx.k_u
    pts = ctx.node_points("viscous", 0)
    vals = inputs.fourier_field(pts.reshape(-1, 3), inputs.fourier_modes(3)).reshape(-1, (k + 1) ** 3, 3)
    uh = torch.tensor(np.ascontiguousarray(vals.transpose(0, 2, 1)).reshape(-1), device="cuda")
    m = 1.5 / dt
    b = ctx.mass("viscous", uh, coeff=m, arith="f64ff")
    rh = inputs.carreau_blood_like()
    out = {"mass_coeff": m}
    for aitken in (True, False):
        u = uh.clone()
        r = ctx.picard_solve(rh, b, u, mass=m, rtol=1e-6, maxit=40, aitken=aitken, lin_rtol=1e-3)
        out["aitken" if aitken else "plain_picard"] = {
            "status": r["status"], "updates": r["iterations"], "cg_iterations": r["lin_iterations"],
            "seconds": r["seconds"], "res0": r["res0"], "res": r["res"],
            "omegas": [round(w, 4) for w in r["omegas"]]}
    return out


def step_extras(n_cells=32, k=3, courant=0.3, warm=2, steps=5):
    """Projection-scheme time steps on a lid-driven box (lid velocity (1, 0, 0)
    on +z, no-slip elsewhere), Carreau-Yasuda viscosity linear implicit, the
    seeded Fourier field as initial velocity, dt from the CFL rule (Cr = 0.3),
    pressure and viscous CG to 1e-8. Host-clock step times (the step
    synchronises); CUDA-event times of the step's form kernels."""
    import numpy as np
    import torch

    from paper_2506_14424_gb300 import Context, inputs
    ctx = Context(n_cells, n_cells, n_cells, k, krylov_arith="f64ff")
    rh = inputs.carreau_blood_like()
    pts = ctx.node_points("viscous", 0)
    vals = inputs.fourier_field(pts.reshape(-1, 3), inputs.fourier_modes(1)).reshape(-1, (k + 1) ** 3, 3)
    u0 = torch.tensor(np.ascontiguousarray(vals.transpose(0, 2, 1)).reshape(-1), device="cuda")
    wall = np.zeros((6, 3))
    wall[5, 0] = 1.0
    out = {"n_dofs_velocity": ctx.n_dofs("viscous"), "n_dofs_pressure": ctx.n_dofs("poisson")}

    def ev(fn, reps=10):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        for _ in range(reps):
            fn()
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    y = torch.empty_like(u0)
    p = torch.tensor(inputs.uniform_vector(ctx.n_dofs("poisson"), 3), device="cuda")
    out["convective_ms"] = ev(lambda: ctx.convective(u0, wall, y))
    out["projection_rhs_ms"] = ev(lambda: ctx.projection_rhs(p))
    out["inverse_mass_f64ff_ms"] = ev(lambda: ctx.mass("viscous", u0, y, coeff=2.0, arith="f64ff", inverse=True))
    dt = ctx.cfl_dt(u0, courant)
    out["dt"] = dt
    ctx.step_init(u0)
    rows = []
    for i in range(warm + steps):
        st = ctx.step(rh, dt, wall=wall, ppe_rtol=1e-8, visc_rtol=1e-8)
        if i >= warm:
            rows.append(st)
    keys = ("seconds", "t_convective", "t_pressure", "t_projection", "t_viscous")
    out.update({f"mean_{k2}": float(np.mean([r[k2] for r in rows])) for k2 in keys})
    out["ppe_iterations"] = [r["ppe_iterations"] for r in rows]
    out["visc_iterations"] = [r["visc_iterations"] for r in rows]
    out["steps_per_s"] = 1.0 / out["mean_seconds"]
    # the convective term linearly implicit in the viscous step (alpha_c = 1, GMRES(30)
    # right-preconditioned by the V-cycle), same Courant number
    ctx.step_init(u0)
    rows = []
    for i in range(warm + steps):
        st = ctx.step(rh, dt, wall=wall, ppe_rtol=1e-8, visc_rtol=1e-8, convective_mode="linear_implicit")
        if i >= warm:
            rows.append(st)
    out["linear_implicit_convection"] = {
        "mean_seconds": float(np.mean([r["seconds"] for r in rows])),
        "mean_t_viscous": float(np.mean([r["t_viscous"] for r in rows])),
        "gmres_iterations": [r["visc_iterations"] for r in rows]}
    # explicit convection, ending each step with the divergence and continuity penalty step
    ctx.step_init(u0)
    rows = []
    for i in range(warm + steps):
        st = ctx.step(rh, dt, wall=wall, ppe_rtol=1e-8, visc_rtol=1e-8, penalty=True)
        if i >= warm:
            rows.append(st)
    out["with_penalty_step"] = {
        "mean_seconds": float(np.mean([r["seconds"] for r in rows])),
        "mean_t_penalty": float(np.mean([r["t_penalty"] for r in rows])),
        "penalty_iterations": [r["penalty_iterations"] for r in rows]}
    td, tc = ctx.penalty_tau(u0, dt)
    out["penalty_apply_ms"] = ev(lambda: ctx.penalty_apply(td, tc, u0))
    ctx.close()
    return out


def channel_extras(cells_per_unit=8, k=3, courant=0.3, warm=2, steps=10, t_ramp=1.0, jitter=False, setup_lag=1):
    """Projection-scheme steps on the backward-facing-step channel (inlet [-5, 0] x [1, 2],
    outlet [0, 30] x [0, 2], z in [0, 4] periodic, step height 1, expansion ratio 2), cubes
    of side 1/8: 133,120 hexes, k = 3 velocity / k = 2 pressure; with jitter the vertices
    inside the fluid move by U(-0.05 h, 0.05 h)^3 (seed 4: trilinear cells, FP64 Krylov
    operator), else affine cells (float-float Krylov operator). Parabolic inflow
    of maximum 1 ramped by sin^2(pi t / (2 t_ramp)), traction-free outflow at p = 0, no-slip
    walls and step, Carreau-Yasuda viscosity linear implicit, fluid at rest at t = 0,
    dt from the CFL rule (Cr = 0.3) at the full inflow velocity, CG to 1e-8 with the FP32
    hp-multigrid (p: 3 -> 2 -> 1, then h down to cubes of side 1). The wall data of every
    step are evaluated before the timed steps. Host-clock step times (the step synchronises).
    setup_lag > 1 rebuilds the multigrid eigenvalue estimates and coarse inverse at every
    setup_lag-th viscosity update only (sipg_opts.mg_setup_lag)."""
    import numpy as np
    import torch

    from paper_2506_14424_gb300 import Context, inputs
    c = inputs.bfs_channel(cells_per_unit)
    t0 = time.perf_counter()
    ctx = Context(*c["dims"], k, extent=c["extent"], origin=c["lo"], active=c["active"], periodic=c["periodic"],
                  bc_velocity="DNDDDD", bc_pressure="NDNNNN", bc_removed="DN",
                  krylov_arith="f64" if jitter else "f64ff", coarse_max_dofs=8000, mg_precision="f32",
                  vertices=inputs.bfs_vertices(c) if jitter else None, mg_setup_lag=setup_lag)
    t_create = time.perf_counter() - t0
    rh = inputs.carreau_blood_like()
    n = ctx.n_dofs("viscous")
    ids = torch.tensor(ctx.boundary_faces()[:, 2], device="cuda")
    pts = ctx.boundary_points()
    shape = torch.zeros_like(pts)
    inlet = ids == 0
    shape[inlet, :, 0] = 1.0 - ((pts[inlet, :, 1] - 1.5) / 0.5) ** 2
    dt = courant / k ** 1.5 / (1.0 * cells_per_unit)
    ramp = [float(np.sin(np.pi * (i * dt) / (2 * t_ramp)) ** 2) if i * dt < t_ramp else 1.0
            for i in range(warm + steps + 1)]
    walls = [r * shape for r in ramp]
    ctx.step_init(torch.zeros(n, dtype=torch.float64, device="cuda"))
    rows = []
    for i in range(warm + steps):
        st = ctx.step(rh, dt, wall_points=walls[i + 1], wall_points_prev=walls[i], ppe_rtol=1e-8, visc_rtol=1e-8)
        if i >= warm:
            rows.append(st)
    u = ctx.step_field("u")
    levels = [(tuple(ctx.level_info("viscous", l)[0]), ctx.level_info("viscous", l)[1], ctx.level_info("viscous", l)[2])
              for l in range(ctx.num_levels("viscous"))]
    out = {"geometry": ("trilinear cells (5 % vertex jitter inside the fluid, seed 4)" if jitter
                        else "affine cells (no vertex jitter)"),
           "multigrid": "FP32 V-cycle, FP64 CG", "mg_setup_lag": setup_lag, "cells": ctx.n_cells,
           "n_dofs_velocity": n,
           "n_dofs_pressure": ctx.n_dofs("poisson"), "dt": dt,
           "steps_timed": steps, "create_seconds": t_create, "viscous_levels": levels,
           "mean_seconds": float(np.mean([r["seconds"] for r in rows])),
           "mean_t_pressure": float(np.mean([r["t_pressure"] for r in rows])),
           "mean_t_viscous": float(np.mean([r["t_viscous"] for r in rows])),
           "ppe_iterations": [r["ppe_iterations"] for r in rows],
           "visc_iterations": [r["visc_iterations"] for r in rows],
           "max_u": u.abs().max().item()}
    out["dof_steps_per_s"] = n / out["mean_seconds"]
    ctx.close()
    return out


def trilinear_extras(n_cells=32, k=3, reps=10):
    """Viscous apply (FP64) on trilinear cells: the box's interior vertices jittered by
    U(-0.05 h, 0.05 h)^3 (seed 4, the channel-mesh recipe), Carreau-Yasuda viscosity,
    rotating x/y pairs; the same mesh without jitter through the affine kernel beside it."""
    import numpy as np
    import torch

    from paper_2506_14424_gb300 import Context, inputs
    N = n_cells
    h = 1.0 / N
    g = np.linspace(0.0, 1.0, N + 1)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    V = np.stack([X, Y, Z], axis=-1)
    J = np.random.default_rng(4).uniform(-0.05 * h, 0.05 * h, size=V.shape)
    J[[0, -1], :, :] = 0.0
    J[:, [0, -1], :] = 0.0
    J[:, :, [0, -1]] = 0.0
    out = {}
    for name, verts in (("trilinear", V + J), ("affine", None)):
        ctx = Context(N, N, N, k, vertices=verts)
        n = ctx.n_dofs("viscous")
        ctx.set_viscosity(inputs.carreau_blood_like(), torch.tensor(inputs.uniform_vector(n, 1), device="cuda"))
        xs = [torch.tensor(inputs.uniform_vector(n, seed=100 + i), device="cuda") for i in range(4)]
        ys = [torch.empty_like(xs[0]) for _ in range(4)]
        for i in range(3):
            ctx.apply("viscous", xs[i % 4], ys[i % 4], arith="f64")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        for i in range(reps):
            ctx.apply("viscous", xs[i % 4], ys[i % 4], arith="f64")
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms": ms, "gdofs": n / ms / 1e6}
        if verts is not None:
            # FP32 level applies of the mixed-precision V-cycle on the same cells: the
            # viscous p-levels k = 3, 2, 1 and the pressure level k = 2
            lv = []
            for op, level in (("viscous", 0), ("viscous", 1), ("viscous", 2), ("poisson", 0)):
                _, kl, nd = ctx.level_info(op, level)
                x32 = [torch.tensor(inputs.uniform_vector(nd, seed=200 + i), dtype=torch.float32, device="cuda")
                       for i in range(4)]
                y32 = [torch.empty_like(x32[0]) for _ in range(4)]
                for i in range(3):
                    ctx.apply(op, x32[i % 4], y32[i % 4], level=level)
                e0.record(ctx.stream)
                for i in range(reps):
                    ctx.apply(op, x32[i % 4], y32[i % 4], level=level)
                e1.record(ctx.stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                lv.append({"op": op, "level": level, "k": kl, "n_dofs": nd, "ms": ms, "gdofs": nd / ms / 1e6})
            out[name]["f32_levels"] = lv
        ctx.close()
    # FP64 hp-multigrid CG on the jittered 16^3, k = 3 mesh (h-levels from every other vertex)
    M = 16
    gm = np.linspace(0.0, 1.0, M + 1)
    Zm, Ym, Xm = np.meshgrid(gm, gm, gm, indexing="ij")
    Vm = np.stack([Xm, Ym, Zm], axis=-1)
    Jm = np.random.default_rng(4).uniform(-0.05 / M, 0.05 / M, size=Vm.shape)
    Jm[[0, -1], :, :] = 0.0
    Jm[:, [0, -1], :] = 0.0
    Jm[:, :, [0, -1]] = 0.0
    ctx = Context(M, M, M, k, vertices=Vm + Jm)
    n = ctx.n_dofs("viscous")
    ctx.set_viscosity(inputs.carreau_blood_like(), torch.tensor(inputs.uniform_vector(n, 1), device="cuda"))
    b = torch.tensor(inputs.uniform_vector(n, 2), device="cuda")
    ctx.solve("viscous", b, rtol=1e-8, maxit=500, precond="mg")
    _, st = ctx.solve("viscous", b, rtol=1e-8, maxit=500, precond="mg")
    out["mg_cg_16cubed_k3"] = {"levels": ctx.num_levels("viscous"), "iterations": st["iterations"],
                               "seconds": st["seconds"], "rel_residual": st["rel_residual"]}
    ctx.close()
    return out


def component_timings(stream, contrast=1e2):
    """Each hot-path row on the 16^3, k = 4 sphere workload (CUDA events on the
    context stream; host-synchronous calls timed with the host clock)."""
    import torch

    from paper_2506_14424_gb300 import Context, inputs

    c = Context(16, 16, 16, 4, mg_cph=False)  # the DG levels: one row per p- and h-level
    sink = inputs.sinker(seed=2, count=8, radius=0.1, nu_max=contrast)
    t0 = time.perf_counter()
    c.set_viscosity(sink)
    torch.cuda.synchronize()
    out = {"hierarchy": "dg", "set_viscosity_and_mg_setup_s": time.perf_counter() - t0}

    def ev_time(fn, reps=10):
        for _ in range(2):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    levels = []
    for lvl in range(c.num_levels("viscous")):
        (nx, ny, nz), k, nd = c.level_info("viscous", lvl)
        x64 = torch.tensor(inputs.uniform_vector(nd, seed=60 + lvl), device="cuda")
        y64 = torch.empty_like(x64)
        x32, y32 = x64.float(), y64.float()
        row = {"cells": nx, "k": k, "n_dofs": nd,
               "apply_f64_ms": ev_time(lambda: c.apply("viscous", x64, y64, level=lvl)),
               "apply_f32_ms": ev_time(lambda: c.apply("viscous", x32, y32, level=lvl))}
        if lvl + 1 < c.num_levels("viscous"):
            xs = torch.zeros_like(x32)
            row["smoother_f32_ms"] = ev_time(lambda: c.smooth("viscous", lvl, x32, xs), reps=5)
            row["restrict_f32_ms"] = ev_time(lambda: c.transfer("viscous", lvl, -1, x32))
            ncoarse = c.n_dofs("viscous", lvl + 1)
            xc = torch.zeros(ncoarse, dtype=torch.float32, device="cuda")
            row["prolong_f32_ms"] = ev_time(lambda: c.transfer("viscous", lvl, +1, xc))
        levels.append(row)
    out["levels"] = levels
    b = torch.tensor(inputs.uniform_vector(c.n_dofs(), seed=70), device="cuda")
    out["vcycle_f32_ms"] = ev_time(lambda: c.vcycle("viscous", b), reps=5)
    c.close()
    c = Context(16, 16, 16, 4)  # the default hierarchy on a box (cph)
    t0 = time.perf_counter()
    c.set_viscosity(sink)
    torch.cuda.synchronize()
    out["cph"] = {"set_viscosity_and_mg_setup_s": time.perf_counter() - t0,
                  "levels": c.num_levels("viscous"),
                  "vcycle_f32_ms": ev_time(lambda: c.vcycle("viscous", b), reps=5)}
    c.close()
    return out


def serving_extras(n_req=32, rates=(20.0, 100.0), seed=5, sizes=(8, 12, 16), degrees=(2, 3, 4),
                   contrasts=(1.0, 1e2, 1e4), rhs="buoyancy", budget_gib=96, slots=8, progress=False):
    """Served stream: Poisson arrivals, uneven sizes/degrees/contrasts, rtol 1e-8.

    Each request solves the viscous system on the n^3 unit cube (Dirichlet walls) with
    the sphere ("sinker") viscosity of its contrast (8 spheres of radius 0.15, seed
    1000 + i) and the buoyancy load b = M f of those spheres (f = -e_z inside them).
    The server admits by HBM budget, runs one FP64 CG iteration per request and round
    (FP64 operator, FP32 hp-multigrid V-cycle) with the fine-level applies of each degree
    batched into one launch. The one-at-a-time baseline solves the same requests one
    after another with the same solver (FP64 CG, FP32 hp-multigrid, one context per
    request, no batching; the right-hand side is built outside its service time): its
    service times are measured once and queued against each rate's arrival times
    (FIFO). Latency = completion - arrival."""
    import numpy as np
    import torch

    from paper_2506_14424_gb300 import Context, Server, inputs

    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n_req):
        specs.append({"n": int(rng.choice(sizes)), "k": int(rng.choice(degrees)),
                      "contrast": float(rng.choice(contrasts)), "seed": 1000 + i})
    out = {"requests": n_req, "mix": f"n^3 cells n in {list(sizes)}, k in {list(degrees)}, sphere contrast "
                                     f"{list(contrasts)}, {rhs} right-hand sides, rtol 1e-8",
           "n_dofs_total": int(sum(3 * sp["n"] ** 3 * (sp["k"] + 1) ** 3 for sp in specs))}

    def sinker(sp):
        return inputs.sinker(seed=sp["seed"], count=8, radius=0.15, nu_max=sp["contrast"])

    # one-at-a-time FP64 service times
    service = []
    for sp in specs:
        t0 = time.perf_counter()
        c = Context(sp["n"], sp["n"], sp["n"], sp["k"], mg_precision="f32", krylov_arith="f64")
        c.set_viscosity(sinker(sp))
        nn = c.n_dofs()
        torch.cuda.synchronize()
        tb = time.perf_counter()  # the right-hand side is built outside the service time
        if rhs == "buoyancy":
            f = torch.zeros(nn, dtype=torch.float64, device="cuda").view(-1, 3, (sp["k"] + 1) ** 3)
            pts = torch.tensor(c.node_points("viscous", 0).reshape(-1, (sp["k"] + 1) ** 3, 3), device="cuda")
            cen = torch.tensor(np.asarray(sinker(sp)["centers"]), device="cuda")
            inside = torch.zeros(pts.shape[:2], dtype=torch.bool, device="cuda")
            for ci in range(cen.shape[0]):
                inside |= ((pts - cen[ci]) ** 2).sum(-1) <= 0.15 ** 2
            f[:, 2] = -inside.double()
            b = c.mass("viscous", f.reshape(-1))
        else:
            b = c.apply("viscous", torch.tensor(inputs.uniform_vector(nn, seed=sp["seed"]), device="cuda"))
        torch.cuda.synchronize()
        t_rhs = time.perf_counter() - tb
        c.solve("viscous", b, rtol=1e-8, precond="mg", maxit=400, check=False)
        torch.cuda.synchronize()
        c.close()
        service.append(time.perf_counter() - t0 - t_rhs)
    out["one_at_a_time_service_s"] = {"total": float(sum(service)), "mean": float(np.mean(service)),
                                      "max": float(max(service))}
    if progress:
        print(json.dumps({"serving_one_at_a_time": out["one_at_a_time_service_s"]}), file=sys.stderr, flush=True)
    runs = []
    for rate in rates:
        arr = np.cumsum(np.random.default_rng(seed + int(rate)).exponential(1.0 / rate, n_req))
        # FIFO one-at-a-time baseline against the same arrivals
        fin, lat_seq = 0.0, []
        for a_t, s_t in zip(arr, service):
            fin = max(fin, a_t) + s_t
            lat_seq.append(fin - a_t)
        srv = Server(int(budget_gib) << 30, max_slots=slots)
        t0 = time.perf_counter()
        ids = []
        for sp, a_t in zip(specs, arr):
            dt = t0 + a_t - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            ids.append(srv.submit(sp["n"], sp["k"], sinker(sp), rtol=1e-8, maxit=400, seed=sp["seed"], rhs=rhs))
        srv.drain(3600)
        t_end = time.perf_counter()
        res = [srv.poll(i)[0] for i in ids]
        srv.close()
        lat = np.array([r["latency_s"] for r in res])
        ok = sum(1 for r in res if r["status"] == 0 and r["rel_residual"] <= 1e-8)
        status_counts = {}
        for r in res:
            status_counts[str(r["status"])] = status_counts.get(str(r["status"]), 0) + 1
        runs.append({"rate_per_s": rate, "solves_per_s": n_req / (t_end - t0), "p50_s": float(np.percentile(lat, 50)),
                     "p99_s": float(np.percentile(lat, 99)), "converged": ok, "status_counts": status_counts,
                     "max_rel_residual": max(r["rel_residual"] for r in res),
                     "makespan_s": t_end - t0,
                     "one_at_a_time": {"solves_per_s": n_req / max(fin, arr[-1]),
                                       "p50_s": float(np.percentile(lat_seq, 50)),
                                       "p99_s": float(np.percentile(lat_seq, 99))}})
        if progress:  # one line per finished rate on stderr (long runs)
            print(json.dumps({"serving_rate_done": runs[-1]}), file=sys.stderr, flush=True)
    out["runs"] = runs
    return out


def serving_full():
    """The configured stream: 256 requests, 8^3 .. 48^3 cells, k in {2, 3, 4, 5}, contrast
    in {1, 1e2, 1e4}, sphere-buoyancy right-hand sides, Poisson arrivals at 10, 20, 50, 100
    and 200 per second."""
    return serving_extras(n_req=256, rates=(10.0, 20.0, 50.0, 100.0, 200.0), sizes=(8, 16, 24, 32, 40, 48),
                          degrees=(2, 3, 4, 5), budget_gib=160, slots=12, progress=True)


# ------------------------------------------------------------- CPU oracle
def _oracle_chunk(args):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import numpy as np
    sys.path.insert(0, ROOT)
    from oracle.mesh import BoxMesh
    from oracle.sipg import SIPG
    cells, seed = args
    mesh = BoxMesh(N_CELLS, N_CELLS, N_CELLS)
    S = SIPG(mesh, K_U, 3)
    from paper_2506_14424_gb300 import inputs
    need = set(cells)
    for e in cells:
        for f in range(6):
            nb = mesh.neighbor(e, f)
            if nb is not None:
                need.add(nb)
    # velocity on the needed cells only (same Fourier field as the GPU arm)
    u = np.zeros((mesh.n_cells, 3, S.n ** 3))
    modes = inputs.fourier_modes(1)
    for e in need:
        u[e] = inputs.fourier_field(S.node_points(e), modes).T
    nc, nf = S.viscosity_at_points(inputs.carreau_blood_like(), u.reshape(-1), cells=sorted(need))
    x = np.random.default_rng(seed).uniform(-1, 1, S.n_dofs)
    t0 = time.perf_counter()
    S.apply(x, nc, nf, cells=cells)
    return time.perf_counter() - t0, len(cells) * S.n_dofs_cell


def cpu_baseline(sample_cells=1024, workers=None):
    """The oracle as it stands, timed on this host's cores on a sample of cells."""
    import multiprocessing as mp
    import numpy as np
    workers = workers or os.cpu_count() or 1
    rng = np.random.default_rng(7)
    cells = rng.choice(N_CELLS ** 3, size=sample_cells, replace=False)
    chunks = [(sorted(int(c) for c in ch), 9) for ch in np.array_split(cells, workers)]
    ctxm = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctxm.Pool(workers) as pool:
        res = pool.map(_oracle_chunk, chunks)
    wall = time.perf_counter() - t0
    dofs = sum(r[1] for r in res)
    busy = max(r[0] for r in res)
    # one core: DoFs of each worker over its own busy time, averaged over the workers
    per_core = sum(r[1] / r[0] for r in res) / len(res) / 1e9
    return {"value": dofs / busy / 1e9, "unit": "GDoF/s", "cores": workers, "kind": "oracle",
            "single_core_value": per_core,
            "sample": f"{sample_cells} random cells of the 32^3 k=3 apply (rows of y), explicit element "
                      f"blocks rebuilt per cell, {workers} spawn workers; value = DoFs / slowest worker's "
                      f"apply time ({busy:.1f} s; wall incl. setup {wall:.1f} s); single_core_value = mean "
                      f"over the workers of its DoFs / its apply time"}


def run_reference(args):
    """The FP64 oracle on this host's cores, one bounded sample of cells per step."""
    import multiprocessing as mp
    import numpy as np
    rank, world, _ = dist_env()
    if rank != 0:
        return
    workers = os.cpu_count() or 1
    per_step = max(workers, min(256, (2048 // max(1, args.steps + args.warmup)) // workers * workers))
    rng = np.random.default_rng(7)
    ctxm = mp.get_context("spawn")
    rates = []
    with ctxm.Pool(workers) as pool:
        for i in range(args.warmup + args.steps):
            cells = rng.choice(N_CELLS ** 3, size=per_step, replace=False)
            chunks = [(sorted(int(c) for c in ch), 9 + i) for ch in np.array_split(cells, workers)]
            res = pool.map(_oracle_chunk, chunks)
            busy = max(r[0] for r in res)
            if i >= args.warmup:
                rates.append(sum(r[1] for r in res) / busy / 1e9)
    value = statistics.mean(rates)
    ms_step = 1e3 * per_step * 3 * (K_U + 1) ** 3 / (value * 1e9)
    sample = (f"{per_step} random cells of the 32^3 k=3 apply per step (rows of y), explicit element blocks "
              f"rebuilt per cell, {workers} spawn workers; value = DoFs / slowest worker's apply time")
    line = {"metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "cells": [N_CELLS] * 3, "k_u": K_U},
            "cpu_baseline": {"value": value, "unit": "GDoF/s", "kind": "oracle", "cores": workers, "sample": sample},
            "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.extra:
        run_extra(a.extra, steps=a.channel_steps, lag=a.setup_lag)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)
