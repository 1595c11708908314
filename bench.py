"""Benchmark of the overlap hot path on GB300.

Default workload (the dslash-throughput configuration at the paper's
precision): Wilson dslash on a 24^3 x 64 lattice, even/odd layout with both
parities in one launch, links from exp(0.5 i H) + 3 APE steps (alpha 0.6) +
re-unitarisation, Gaussian spinors, FP64 storage and arithmetic, 1 RHS.
One step = one full-lattice D_w application (one kernel launch).

`value` is GFLOP/s of that kernel (1320 flop per site, the hopping term)
divided by the CUDA-event time.  On GB300 the FP64 dslash is bound by the
FP64 pipe, so its roofline is the FMA throughput measured in the same run by
the library's own FMA kernel.  The JSON line also carries algorithmic GB/s,
the FP32 / FP16 / BF16 / double-float and 12-RHS variants (the FP32 one with
its HBM roofline), a small propagator solve (12 point sources to the FP64
true residual 1e-10), an end-to-end figure through the C ABI with host
buffers, the oracle timed on the host cores, and the SM clocks sampled while
timing.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU (torchrun): replicas only, each rank runs the same workload on its own GPU.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (24, 24, 24, 64)
BC = (1.0, 1.0, 1.0, -1.0)
RHO = 1.5
METRIC = "dslash GB/s & GFLOP/s (% HBM roofline); overlap propagator solves/s at res 1e-10"
REAL_BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2, "df64": 8}
FLOP_SITE = 1320
HEADLINE_PREC = "f64"
FP64_NOMINAL_GFLOPS = 1250.0  # GB300 dense FP64, nominal


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


VARIANT_UNIT = {0: "dslash_regs.cu", 1: "dslash_regs.cu", 2: "dslash_regs.cu", 3: "dslash_staged.cu",
                4: "dslash_staged.cu", 5: "dslash_staged.cu", 6: "dslash_multi.cu", 7: "dslash_multi.cu",
                8: "dslash_batched.cu", 9: "dslash_batched.cu", 10: "dslash_pair.cu", 11: "dslash_pair.cu"}


def kernel_sources_sha(var: int = 1) -> str:
    """Hash of the sources of the dslash kernel of launch variant `var`: a DRAM-traffic figure from
    an ncu capture holds only while the kernel it was taken on is unchanged."""
    h = hashlib.sha256()
    for f in (VARIANT_UNIT[var], "dslash_common.cuh", "ov_internal.cuh", "ov_kernels.h"):
        with open(os.path.join(ROOT, "paper_1106_4964_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch, from the ncu captures
# summarised under profiles/, keyed by (kernel, lattice, sources hash at capture time).  A kernel whose
# sources changed since its capture gets null.
NCU_TRAFFIC = {
    # FP64, 1 rhs, block 256 x 1, register-budget variant 1 (the default run's timed kernel)
    ("dslash_kernel<f64,f64,variant=1>", (24, 24, 24, 64), "625052d99d5871d2"): 734_775_552 + 153_691_392,
}


def ncu_traffic(kernel: str, var: int):
    return NCU_TRAFFIC.get((kernel, tuple(DIMS), kernel_sources_sha(var)))


def kernel_name(prec: str, var: int, nrhs: int = 1) -> str:
    """The CUDA kernel a dslash launch of this precision and launch variant runs."""
    if var == 3:
        return f"dslash_staged_kernel<{prec},{prec}>"
    if var in (4, 5):
        return f"dslash_tma_kernel<{prec},{prec},links_prefetched={var == 5}>"
    if var in (6, 7):
        return f"dslash_multi_kernel<{prec},{prec},rhs_per_thread={2 if var == 6 else 4}>"
    if var in (8, 9):
        return f"dslash_batched_kernel<{prec},{prec},hops_batched={4 if var == 8 else 8}>"
    if var in (10, 11):
        return f"dslash_pair_kernel<{prec},{prec},rhs_pairs_per_thread={1 if var == 10 else 2}>"
    return f"dslash_kernel<{prec},{prec},variant={var}>"


def site_bytes(prec: str, nrhs: int = 1) -> float:
    """Compulsory bytes per site and RHS of a one-pass full D_w: 4 reconstruct-12 links (48 reals)
    shared by the RHS, input and output spinors 24 reals each (16-bit spinors add a 4-byte
    scale).  The FP64 and double-float kernels store all 18 reals of a link (they are bound by
    arithmetic, not bandwidth); the algorithmic figure keeps the 12-real minimum."""
    rb = REAL_BYTES[prec]
    spin = 24 * rb + (4 if prec in ("f16", "bf16") else 0)
    return 48 * rb / nrhs + 2 * spin


def clenshaw_step_bytes(prec: str, nrhs: int, f32_work: bool) -> float:
    """Compulsory bytes per site and RHS of one Clenshaw step (two D_w launches, the second with the
    fused epilogue b_k = c_k psi_h + alpha H_w t + beta b_{k+1} - b_{k+2}): twice the D_w bytes plus the
    three epilogue fields.  16-bit storage with FP32 recurrence fields (the library's default) moves
    FP32 spinors and 16-bit links."""
    work = "f32" if (prec in ("f16", "bf16") and f32_work) else prec
    rb = REAL_BYTES[work]
    spin = 24 * rb + (4 if work in ("f16", "bf16") else 0)
    links = 48 * REAL_BYTES[prec] / nrhs
    return 2 * (links + 2 * spin) + 3 * spin


class Clocks:
    """Samples nvidia-smi every 200 ms in the background."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r for r in self.rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_inputs(nrhs=1):
    import synth

    U = synth.gauge_field(DIMS, seed=1, s=0.5, ape_steps=3)
    psi = synth.gaussian_spinor(DIMS, seed=2, nrhs=nrhs)
    return U, psi


def time_dslash(ctx, psi_dev, prec, nrhs, steps, warmup, torch):
    """Average CUDA-event time of one D_w launch (internal fields, current stream) in the
    autotuned launch shape; returns (ms, (bx, by, variant))."""
    fi, fo = ctx.field(nrhs, prec), ctx.field(nrhs, prec)
    fi.load(psi_dev)
    shape = ctx.tune_dslash(prec, nrhs)
    st = torch.cuda.current_stream()
    for _ in range(warmup):
        ctx.dslash_field(fi, fo, -RHO)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        ctx.dslash_field(fi, fo, -RHO)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    fi.close()
    fo.close()
    return ms, shape


def dslash_config(world: int = 1, prec: str = HEADLINE_PREC, nrhs: int = 1) -> dict:
    """The headline workload, the same for the GPU arm and the oracle (reference) arm."""
    if prec == HEADLINE_PREC and nrhs == 1:
        what = "FP64 storage and arithmetic (the paper's precision), 1 rhs"
    else:
        what = f"{prec} storage, {nrhs} rhs (profiling run, not the headline)"
    return {"workload": f"wilson dslash D_w, 24^3x64 even/odd, {what}, both parities per launch",
            "lattice": list(DIMS), "gauge": "exp(0.5 iH) + 3 APE(0.6) steps", "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2: gauge 510 MB + spinors 2 x 170 MB per launch"}


def replica_time(ms: float, dist, device: str) -> float:
    """The job's time per step under replicas: the maximum over ranks (the slowest replica)."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput: the units every rank processed in the job's time (units per second)."""
    return units_per_rank * world / (ms * 1e-3)


def run_gpu(args):
    import torch

    import paper_1106_4964_gb300 as ov

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    V = int(np.prod(DIMS))
    U, psi = make_inputs(1)
    ctx = ov.Context(DIMS, BC)
    U_dev = torch.from_numpy(U).cuda()
    ctx.set_gauge(U_dev)
    psi_dev = torch.from_numpy(psi).cuda()
    hbm, peak_kind = peaks()
    # ALU rooflines: FMA throughput of this GPU, measured by the library's own FMA kernel
    fma = {"f64_gflops": round(ov.measure_fma_peak("f64"), 1), "f32_gflops": round(ov.measure_fma_peak("f32"), 1),
           "how": "ov_measure_fma_peak: 8 independent FMA chains per thread, 8 x 256 threads per SM, "
                  "best of 5 launches (CUDA events), 2 flop per FMA"}

    # ---- headline: FP64, 1 rhs (timed region bracketed by barrier + synchronize); --prec / --nrhs
    # select another launch of the same lattice for profiling runs
    prec, nrhs = args.prec, args.nrhs
    if nrhs > 1:
        psi_dev = torch.from_numpy(make_inputs_rhs(nrhs)).cuda()
    fi, fo = ctx.field(nrhs, prec), ctx.field(nrhs, prec)
    fi.load(psi_dev)
    if args.shape:
        bx, by, var = args.shape
        ctx.set_dslash_shape(prec, nrhs, bx, by, var)
    else:
        bx, by, var = ctx.tune_dslash(prec, nrhs)
    st = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ctx.dslash_field(fi, fo, -RHO)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, int(args.inner))
    n0 = ctx.dslash_count()
    t_wall = time.perf_counter()
    e0.record(st)
    for _ in range(args.steps * reps):
        ctx.dslash_field(fi, fo, -RHO)
    e1.record(st)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    launches = ctx.dslash_count() - n0
    if dist:
        dist.barrier()
    time.sleep(0.3)
    clocks = clk.stop()
    ms = replica_time(e0.elapsed_time(e1) / (args.steps * reps), dist, "cuda")
    bytes_launch = V * nrhs * site_bytes(prec, nrhs)
    gbs = bytes_launch / (ms * 1e-3) / 1e9
    gflops = FLOP_SITE * V * nrhs / (ms * 1e-3) / 1e9
    fi.close()
    fo.close()
    if nrhs > 1:
        psi_dev = torch.from_numpy(psi).cuda()

    # ---- variants (same lattice, other precisions and 12 rhs); the FP32 one is bound by HBM
    variants = {}
    if not args.quick:
        for p in ("f32", "f16", "bf16", "df64"):
            t, sh = time_dslash(ctx, psi_dev, p, 1, min(2000, max(20, args.steps)), args.warmup, torch)
            b = V * site_bytes(p, 1)
            variants[f"{p}_r1"] = {"ms": round(t, 4), "GBps": round(b / t / 1e6, 1),
                                   "GFLOPps": round(FLOP_SITE * V / t / 1e6, 1),
                                   "frac_hbm": round(b / t / 1e6 / hbm, 3), "kernel": kernel_name(p, sh[2]),
                                   "shape": list(sh)}
        variants["df64_r1"]["frac_f32_fma_note"] = "double-float is bound by the FP32 pipe, not HBM"
        psi12 = torch.from_numpy(make_inputs_rhs(12)).cuda()
        for p in ("f32", "f16", "f64", "df64"):
            t, sh = time_dslash(ctx, psi12, p, 12, min(300, max(5, args.steps // 2)), args.warmup, torch)
            b = V * 12 * site_bytes(p, 12)
            variants[f"{p}_r12"] = {"ms": round(t, 4), "GBps": round(b / t / 1e6, 1),
                                    "GFLOPps": round(12 * FLOP_SITE * V / t / 1e6, 1),
                                    "frac_hbm": round(b / t / 1e6 / hbm, 3), "kernel": kernel_name(p, sh[2], 12),
                                    "shape": list(sh), "ms_per_rhs": round(t / 12, 4)}
        del psi12

    # ---- end to end through the C ABI with pinned host buffers (H2D + pack + dslash + unpack + D2H)
    hin = torch.from_numpy(psi).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    for _ in range(2):
        ctx.apply_dslash(hin.numpy(), hout.numpy(), -RHO, prec=prec)
    torch.cuda.synchronize()
    ne = min(10, max(3, args.steps // 4))
    t0 = time.perf_counter()
    for _ in range(ne):
        ctx.apply_dslash(hin.numpy(), hout.numpy(), -RHO, prec=prec)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / ne
    e2e = {"value": round(FLOP_SITE * V / e2e_s / 1e9, 2), "unit": "GFLOP/s",
           "h2d_bytes_per_step": int(hin.numel() * hin.element_size()),
           "d2h_bytes_per_step": int(hout.numel() * hout.element_size()),
           "ms_per_step": round(e2e_s * 1e3, 3)}
    ctx.close()
    del U_dev, psi_dev
    torch.cuda.empty_cache()

    prop = None
    if not args.quick and not args.no_prop and rank == 0:
        try:
            prop = propagator_record(args)
        except Exception as e:  # the headline stands on its own: record the failure instead of losing the line
            prop = {"error": f"{type(e).__name__}: {e}"}

    kern = kernel_name(prec, var, nrhs)
    fma_peak = fma["f64_gflops"] if prec == "f64" else fma["f32_gflops"]
    out = {
        "metric": METRIC,
        "value": round(replica_throughput(FLOP_SITE * V * nrhs / 1e9, world, ms), 2),
        "unit": "GFLOP/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms * reps, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": prec,
        "data": "synthetic",
        "config": dict(dslash_config(world, prec, nrhs), launch_shape=[bx, by], variant=var,
                       launches_per_step=reps),
        "GBps": round(gbs * world, 1),
        "roofline": {"bound": "alu", "achieved": round(gflops, 1), "peak": fma_peak, "unit": "GFLOP/s",
                     "frac": round(gflops / fma_peak, 4), "traffic": ncu_traffic(kern, var),
                     "peak_kind": f"measured: {prec if prec in ('f64', 'f32') else 'f32'} FMA throughput of this "
                                  "GPU (ov_measure_fma_peak, same run)",
                     "peak_nominal": FP64_NOMINAL_GFLOPS, "frac_nominal": round(gflops / FP64_NOMINAL_GFLOPS, 4),
                     "algorithmic_flops_per_launch": FLOP_SITE * V, "kernel": kern,
                     "hbm": {"achieved": round(gbs, 1), "peak": hbm, "frac": round(gbs / hbm, 4),
                             "peak_kind": peak_kind, "algorithmic_bytes_per_launch": int(bytes_launch)}},
        "fma_peaks": fma,
        "variants": variants,
        "propagator": prop,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "wall_s_timed": round(t_wall, 4),
    }
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(U, psi, args)
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def sign_for_delta(ctx, eps, lmax, delta, degree):
    """Install the Chebyshev sign on [eps, 1] with the lowest degree (a multiple of 10, at most 1000)
    whose accuracy delta (Eq. 4, as the library evaluates it) is at most `delta`; a fixed `degree`
    when delta is 0.  Returns (degree, delta)."""
    if not delta > 0:
        ctx.set_sign_poly(RHO, eps, degree, lmax)
        return degree, ctx.get_option("sign_delta")
    lo, hi = 1, 100  # bisection on multiples of 10: delta(10 lo) > target, delta(10 hi) <= target (or hi = 100)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        ctx.set_sign_poly(RHO, eps, 10 * mid, lmax)
        if ctx.get_option("sign_delta") <= delta:
            hi = mid
        else:
            lo = mid
    ctx.set_sign_poly(RHO, eps, 10 * hi, lmax)
    return 10 * hi, ctx.get_option("sign_delta")


def propagator_record(args):
    """A small propagator at the paper's precision, inside the default run: the 12 spin-colour point
    sources on an 8^3 x 16 lattice (the same link generator), rho 1.5, the lowest 16 H_w modes deflated
    in the sign (on the rest, the lowest Chebyshev degree with delta <= 1e-10, the accuracy the paper
    tunes its polynomial to) and the lowest 16 D^dag D modes deflating the CG, one
    multi-RHS mixed-precision CG (FP32 inner operator on the chiral sectors, FP64 true residuals and
    reliable updates) to the FP64 true residual 1e-10, quark mass --prop-mass.  Set-up (eigensolvers)
    is timed apart."""
    import torch

    import paper_1106_4964_gb300 as ov
    import synth

    dims = tuple(args.prop_dims)
    U = synth.gauge_field(dims, seed=1, s=0.5, ape_steps=3)
    ctx = ov.Context(dims, BC)
    ctx.set_gauge(torch.from_numpy(U).cuda())
    ctx.set_option("hi_prec", ov.PREC["f64"])
    setup = {}
    t0 = time.perf_counter()
    ctx.set_sign_poly(RHO, 0.05, 100, 0.0)
    lmax = ctx.get_sign_poly()["lambda_max"]
    ctx.deflate(0, args.prop_nev, 1e-8)
    vals, _ = ctx.get_eigenpairs(0)
    eps = (0.99 * np.abs(vals).max() / lmax) ** 2
    degree, delta = sign_for_delta(ctx, eps, lmax, 1e-10, 0)
    setup["deflate_hw"] = time.perf_counter() - t0
    ctx.set_option("chiral", 1)
    t0 = time.perf_counter()
    ctx.deflate(1, args.prop_nev, 1e-8)
    setup["deflate_dd"] = time.perf_counter() - t0
    ctx.tune_dslash("f32", 12)
    b = torch.from_numpy(synth.point_sources(dims)).cuda()
    x = torch.empty_like(b)
    n0 = ctx.dslash_count()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = ctx.cg_solve(b, x, mass=args.prop_mass, tol=1e-10, max_iter=3000, inner_prec="f32")
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    rec = {"workload": f"12 point sources, {dims[0]}^3x{dims[3]}, rho 1.5, mass {args.prop_mass}, {args.prop_nev} H_w + "
                       f"{args.prop_nev} D^dag D modes, degree {degree} (delta {delta:.2g}), eps {eps:.4g}",
           "solves_per_s": round(12 / t, 4), "propagators_per_s": round(1 / t, 5), "seconds": round(t, 3),
           "iterations": info["iterations"], "reliable_updates": info["reliable_updates"],
           "fallback": info["fallback"],
           "max_fp64_true_residual": max(info["true_residual"]), "dslash_launches": ctx.dslash_count() - n0,
           "graphs": list(ctx.graph_stats()), "setup_s": {k: round(v, 2) for k, v in setup.items()},
           "method": "FP32 inner operator (one-sign chiral form), FP64 true residuals and reliable updates"}
    ctx.close()
    return rec


def make_inputs_rhs(nrhs):
    import synth

    return synth.gaussian_spinor(DIMS, seed=3, nrhs=nrhs)


def cpu_baseline(U, psi, args):
    """The FP64 oracle (plain C, OpenMP over all host cores) on a bounded sample of the same
    workload: whole D_w applications of the 24^3 x 64 lattice until ~10 s have passed."""
    import oracle

    oracle.build()
    V = int(np.prod(DIMS))
    t0 = time.perf_counter()
    n = 0
    while True:
        oracle.dslash(DIMS, BC, U, -RHO, psi[0])
        n += 1
        if time.perf_counter() - t0 > args.cpu_seconds:
            break
    dt = (time.perf_counter() - t0) / n
    cores = oracle.threads()
    # one core: a single application (about 16x the all-core time)
    oracle.set_threads(1)
    t1 = time.perf_counter()
    oracle.dslash(DIMS, BC, U, -RHO, psi[0])
    dt1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    return {"value": round(FLOP_SITE * V / dt / 1e9, 3), "unit": "GFLOP/s", "cores": cores,
            "kind": "oracle", "GBps": round(V * site_bytes("f64", 1) / dt / 1e9, 3),
            "one_core": {"value": round(FLOP_SITE * V / dt1 / 1e9, 3), "unit": "GFLOP/s"},
            "sample": f"{n} full D_w applications of the 24^3x64 lattice (FP64 oracle), {dt * 1e3:.1f} ms each "
                      f"on {cores} threads, one more on 1 thread ({dt1 * 1e3:.0f} ms)"}


def cpu_dw_extrapolation(U, dims, launches, args):
    """Oracle estimate of one solve: the FP64 oracle's D_w timed on this lattice (whole
    applications for about --cpu-seconds), times the D_w applications per source of the GPU
    solve (each multi-RHS launch applies D_w once per right-hand side).  Vector updates and
    projections are left out, so the estimate favours the CPU."""
    import oracle
    import synth

    oracle.build()
    psi = synth.gaussian_spinor(dims, seed=2, nrhs=1)[0]
    t0 = time.perf_counter()
    n = 0
    while True:
        oracle.dslash(dims, BC, U, -RHO, psi)
        n += 1
        if time.perf_counter() - t0 > min(args.cpu_seconds, 10.0):
            break
    dt = (time.perf_counter() - t0) / n
    t_solve = dt * launches
    return {"value": round(1.0 / t_solve, 6), "unit": "solves/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{n} FP64 oracle D_w applications on {dims[0]}^3x{dims[3]} ({dt * 1e3:.1f} ms each), "
                      f"extrapolated to the {launches} D_w applications per source of the GPU solve"}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores (rank 0 only), the same D_w on the
    same lattice, in the same unit."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    U, psi = make_inputs(1)
    import oracle

    oracle.build()
    V = int(np.prod(DIMS))
    for _ in range(args.warmup if args.warmup < 2 else 1):
        oracle.dslash(DIMS, BC, U, -RHO, psi[0])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.dslash(DIMS, BC, U, -RHO, psi[0])
    dt = (time.perf_counter() - t0) / args.steps
    cores = oracle.threads()
    val = round(FLOP_SITE * V / dt / 1e9, 3)
    sample = (f"{args.steps} full D_w applications of the 24^3x64 lattice by the FP64 CPU oracle (canonical "
              "layout, plain loops, OpenMP)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dslash_config(args.gpus),
        "cpu_baseline": {"value": val, "unit": "GFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "GBps": round(V * site_bytes("f64", 1) / dt / 1e9, 3)}))


# ---------------------------------------------------------------------------------------
# further workloads (not run by default): the overlap application, the batched
# propagator and the learned preconditioner.  Each prints one JSON line.
# ---------------------------------------------------------------------------------------
def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_overlap(args):
    """Overlap application on 24^3 x 64 (rho 1.5): the lowest nev H_w modes deflated (subspace
    iteration on T_100(H_w^2), FP32 filter, FP64 Gram-Schmidt and Rayleigh-Ritz), degree-n Chebyshev on the rest,
    eps = (0.99 |lambda_nev| / lambda_max)^2.  Times one application per precision (1 and 12 rhs)
    and reports each precision's error against the FP64 application."""
    import torch

    import paper_1106_4964_gb300 as ov

    torch.cuda.set_device(0)
    dims = tuple(args.dims) if args.dims else DIMS
    V = int(np.prod(dims))
    import synth

    U = synth.gauge_field(dims, seed=1, s=0.5, ape_steps=3)
    hbm, _ = peaks()
    ctx = ov.Context(dims, BC)
    ctx.set_gauge(torch.from_numpy(U).cuda())
    t0 = time.perf_counter()
    ctx.set_sign_poly(RHO, 0.05, args.degree, 0.0)
    lmax = ctx.get_sign_poly()["lambda_max"]
    t_lmax = time.perf_counter() - t0
    t0 = time.perf_counter()
    ctx.deflate(0, args.nev, args.eig_tol)
    torch.cuda.synchronize()
    t_defl = time.perf_counter() - t0
    vals, _ = ctx.get_eigenpairs(0)
    eps = (0.99 * np.abs(vals).max() / lmax) ** 2
    ctx.set_sign_poly(RHO, eps, args.degree, lmax)
    psi = torch.from_numpy(synth.gaussian_spinor(dims, seed=2, nrhs=1)).cuda()
    psi12 = torch.from_numpy(synth.gaussian_spinor(dims, seed=3, nrhs=12)).cuda()
    ref = None
    res = {}
    for prec in ("f64", "df64", "f32", "f16", "bf16"):
        for nrhs, src in ((1, psi), (12, psi12)):
            if nrhs == 12 and prec == "f64" and not args.f64_r12:
                continue
            ctx.tune_dslash(prec, nrhs)
            fi, fo = ctx.field(nrhs, prec), ctx.field(nrhs, prec)
            fi.load(src)
            ctx.overlap_field(fi, fo)  # eager run, then capture of the graph that the timed calls replay
            torch.cuda.synchronize()
            n0 = ctx.dslash_count()
            e0, e1 = _events(torch)
            reps = 1 if prec == "f64" else args.reps
            e0.record()
            for _ in range(reps):
                ctx.overlap_field(fi, fo)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            launches = (ctx.dslash_count() - n0) // reps
            out = torch.empty_like(src)
            fo.store(out)
            if prec == "f64" and nrhs == 1:
                ref = out.clone()
            err = None
            if nrhs == 1 and ref is not None:
                err = float(torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref))
            steps = launches / 2.0  # Clenshaw steps (the final D_w launch counted as half a step)
            cb = clenshaw_step_bytes(prec, nrhs, bool(ctx.get_option("clenshaw_f32")))
            gbs = steps * V * nrhs * cb / (ms * 1e-3) / 1e9
            res[f"{prec}_r{nrhs}"] = {"ms": round(ms, 3), "applications_per_s": round(1e3 * nrhs / ms, 3),
                                      "dslash_launches": int(launches), "rel_err_vs_f64": err,
                                      "us_per_launch": round(1e3 * ms / max(1, launches), 2),
                                      "clenshaw_step_GBps": round(gbs, 1), "frac_hbm": round(gbs / hbm, 3)}
            fi.close()
            fo.close()
    main = res["f32_r1"]
    cpu = None
    if not args.no_cpu:
        cpu = cpu_dw_extrapolation(U, dims, 2 * args.degree + 1, args)
        cpu["value"], cpu["unit"] = cpu["value"], "applications/s"
        cpu["sample"] = cpu["sample"].replace("per source of the GPU solve", "of one overlap application")
    print(json.dumps({
        "metric": "overlap applications/s", "value": main["applications_per_s"], "unit": "applications/s",
        "n_gpus": 1, "steps": args.reps, "warmup": 1, "ms_per_step": main["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"overlap D(0) application, {dims[0]}^3x{dims[3]}, rho 1.5, {args.nev} deflated H_w "
                               f"modes, degree {args.degree}", "lattice": list(dims), "eps": eps,
                   "lambda_max": lmax},
        "setup_s": {"lambda_max": round(t_lmax, 2), "deflate": round(t_defl, 2)},
        "eigen": {"nev": int(len(vals)), "min_abs": float(np.abs(vals).min()), "max_abs": float(np.abs(vals).max())},
        "precisions": res, "cpu_baseline": cpu}))


def run_project(args):
    """The low-mode projection of Eq. 7 at 24^3 x 64 with nev seeded orthonormal fields standing in for
    eigenvectors (the contractions do not depend on their values): c = v^dag psi and the update
    psi - v c, gamma5 v (s o c) on the tensor cores (bf16 rows; FP32 fields add the bf16 remainder rows)
    against the CUDA cores, 1 and 12 right-hand sides."""
    import torch

    import paper_1106_4964_gb300 as ov
    import synth

    torch.cuda.set_device(0)
    dims = tuple(args.dims) if args.dims else DIMS
    V = int(np.prod(dims))
    ctx = ov.Context(dims, BC)
    ctx.set_gauge(torch.from_numpy(synth.unit_gauge(dims)).cuda())
    g = torch.Generator(device="cuda").manual_seed(7)
    vecs = torch.randn((args.nev, V * 12), dtype=torch.complex128, device="cuda", generator=g)
    vecs /= torch.linalg.vector_norm(vecs, dim=1, keepdim=True)
    sg = np.where(np.arange(args.nev) % 2 == 0, 1.0, -1.0)
    ctx.set_eigenpairs(0, 0.5 * sg, vecs)
    del vecs
    torch.cuda.empty_cache()
    hbm, _ = peaks()
    out = {}
    K = 24 * V
    for nrhs in (1, 12):
        psi = torch.from_numpy(synth.gaussian_spinor(dims, seed=2, nrhs=nrhs)).cuda()
        for prec in ("f32", "f16"):
            f, o1, o2 = ctx.field(nrhs, prec), ctx.field(nrhs, prec), ctx.field(nrhs, prec)
            f.load(psi)
            coef = ctx.project_lowmodes(0, f, engine=0)
            for name, engines in (("dots", ((2 if prec == "f32" else 1, "tensor_cores"), (0, "cuda_cores"))),
                                  ("update", ((1, "tensor_cores"), (0, "cuda_cores")))):
                for engine, ename in engines:
                    def call():
                        if name == "dots":
                            ctx.project_lowmodes(0, f, engine=engine)
                        else:
                            ctx.lowmode_update(0, f, coef, o1, o2, engine=engine)
                    call()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    for _ in range(args.reps):
                        call()
                    torch.cuda.synchronize()
                    ms = (time.perf_counter() - t0) / args.reps * 1e3
                    # rows: bf16 (2 B) per real for 16-bit fields and 1 split; 4 B (rows + remainders) for FP32
                    # on the tensor cores; the CUDA cores read the rows in the field's precision
                    rb = (4 if prec == "f32" else 2) if engine else (4 if prec == "f32" else 2.17)
                    fb = 4 if prec == "f32" else 2.17
                    bytes_alg = args.nev * K * rb + nrhs * K * fb * (1 if name == "dots" else 3)
                    out[f"{name}_{prec}_{ename}_r{nrhs}"] = {"ms": round(ms, 4), "GBps": round(bytes_alg / ms / 1e6, 1),
                                                             "frac_hbm": round(bytes_alg / ms / 1e6 / hbm, 3)}
            for x in (f, o1, o2):
                x.close()
    print(json.dumps({"metric": "low-mode projection GB/s", "value": out["update_f32_tensor_cores_r1"]["GBps"],
                      "unit": "GB/s", "n_gpus": 1, "steps": args.reps, "warmup": 1,
                      "ms_per_step": out["update_f32_tensor_cores_r1"]["ms"], "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "bf16 x bf16 -> f32", "data": "synthetic",
                      "config": {"workload": f"eta^dag psi and psi - eta c, {args.nev} vectors, {dims}",
                                 "lattice": list(dims),
                                 "timing": "wall clock over the synchronising ABI calls (includes the coefficient "
                                           "copy and the call's synchronisation)"},
                      "results": out}))


def run_propagator(args):
    """Batched propagator: 12 spin-colour point sources at the origin, rho 1.5, the lowest nev H_w
    modes deflated in the sign and the lowest nev_cg modes of D^dag D deflating the CG, mixed-precision
    CG on D^dag D to 1e-10 with FP64 reliable updates, 12 rhs in one multi-RHS launch per dslash,
    graph-captured operator applications, autotuned launch shape."""
    import torch

    import paper_1106_4964_gb300 as ov
    import synth

    torch.cuda.set_device(0)
    dims = tuple(args.dims) if args.dims else (32, 32, 32, 64)
    U = synth.gauge_field(dims, seed=1, s=0.5, ape_steps=3)
    ctx = ov.Context(dims, BC)
    ctx.set_gauge(torch.from_numpy(U).cuda())
    ctx.set_option("reliable_delta", args.delta)
    ctx.set_option("hi_prec", ov.PREC[args.hi_prec])
    setup = {}
    t0 = time.perf_counter()
    ctx.set_sign_poly(RHO, 0.05, args.degree, 0.0)
    lmax = ctx.get_sign_poly()["lambda_max"]
    setup["lambda_max"] = time.perf_counter() - t0
    eps = 0.05
    if args.nev > 0:
        t0 = time.perf_counter()
        ctx.deflate(0, args.nev, args.eig_tol)
        setup["deflate_hw"] = time.perf_counter() - t0
        vals, _ = ctx.get_eigenpairs(0)
        eps = (0.99 * np.abs(vals).max() / lmax) ** 2
    degree, delta = sign_for_delta(ctx, eps, lmax, args.sign_delta, args.degree)
    ctx.set_option("chiral", int(args.chiral))
    if args.nev_cg > 0:
        ctx.set_option("filter_dd", args.filter_dd)
        t0 = time.perf_counter()
        ctx.deflate(1, args.nev_cg, args.eig_tol)
        setup["deflate_dd"] = time.perf_counter() - t0
    b = torch.from_numpy(synth.point_sources(dims)).cuda()
    for p in ("f32", "f16", args.hi_prec):
        ctx.tune_dslash(p, 12)
    def solve(src, inner):
        x = torch.empty_like(src)
        n0 = ctx.dslash_count()
        info = ctx.cg_solve(src, x, mass=args.mass, tol=1e-10, max_iter=args.max_iter, inner_prec=inner)
        nrhs = src.shape[0]
        return {"seconds": round(info["seconds"], 2), "iterations": info["iterations"],
                "reliable_updates": info["reliable_updates"], "dslash_launches": ctx.dslash_count() - n0,
                "max_true_residual": max(info["true_residual"][:nrhs]),
                "solves_per_s": round(nrhs / info["seconds"], 4)}

    out, xs = {}, {}
    for inner in args.cg_inner.split(","):
        x = torch.empty_like(b)
        n0 = ctx.dslash_count()
        info = ctx.cg_solve(b, x, mass=args.mass, tol=1e-10, max_iter=args.max_iter, inner_prec=inner)
        out[inner] = {"seconds": round(info["seconds"], 2), "iterations": info["iterations"],
                      "reliable_updates": info["reliable_updates"], "dslash_launches": ctx.dslash_count() - n0,
                      "max_true_residual": max(info["true_residual"][:12]),
                      "solves_per_s": round(12 / info["seconds"], 4)}
        xs[inner] = x
    best_inner = min(out, key=lambda k: out[k]["seconds"])
    best = out[best_inner]
    xbest = xs[best_inner]
    # the solution checked once with the FP64 operator (two-sign D(m)^dag D(m), FP64 storage and
    # arithmetic), whatever the precision of the solver's own true residuals
    t0 = time.perf_counter()
    Ax = torch.empty_like(b)
    ctx.apply_normal(xbest, Ax, args.mass, prec="f64")
    torch.cuda.synchronize()
    r = (b - Ax).reshape(12, -1)
    fp64_res = (torch.linalg.vector_norm(r, dim=1) / torch.linalg.vector_norm(b.reshape(12, -1), dim=1)).tolist()
    best["fp64_true_residual_max"] = max(fp64_res)
    best["fp64_check_seconds"] = round(time.perf_counter() - t0, 2)
    # the same method one source at a time (no batching), and the plain FP64 method
    compare = {}
    if args.plain_rhs > 0:
        compare[f"unbatched_{best_inner}"] = solve(b[:1], best_inner)
        ctx.set_option("chiral", 0)
        ctx.set_option("hi_prec", ov.PREC["f64"])
        ctx.tune_dslash("f64", args.plain_rhs)
        compare["plain_f64"] = solve(b[:args.plain_rhs], "f64")
        compare["plain_f64"]["note"] = (f"FP64 inner operator and true residuals, full D^dag D, "
                                        f"{args.plain_rhs} of the 12 sources")
    cpu = None
    if not args.no_cpu:
        cpu = cpu_dw_extrapolation(U, dims, best["dslash_launches"], args)
    print(json.dumps({
        "metric": "overlap propagator solves/s at res 1e-10", "value": best["solves_per_s"], "unit": "solves/s",
        "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": round(1e3 * best["seconds"], 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": f"mixed {args.cg_inner.replace(',', '/')} + {args.hi_prec}",
        "data": "synthetic",
        "config": {"workload": f"12 point sources, {dims[0]}^3x{dims[3]}, rho 1.5, mass {args.mass}, "
                               f"{args.nev} H_w modes + {args.nev_cg} D^dag D modes, degree {degree}",
                   "lattice": list(dims), "eps": eps, "lambda_max": lmax, "sign_delta": delta,
                   "hi_prec": args.hi_prec,
                   "chiral": bool(args.chiral)},
        "propagators_per_s": round(best["solves_per_s"] / 12, 5),
        "setup_s": {k: round(v, 1) for k, v in setup.items()}, "solves": out, "compare": compare,
        "cpu_baseline": cpu}))


def run_learned(args):
    """Learned preconditioner: train on (residual, error) pairs of deflated CG solves on a small
    lattice, move the weights to the large lattice, and compare flexible CG with plain deflated
    CG on 12 sources (iterations and time to 1e-10)."""
    import torch

    import paper_1106_4964_gb300 as ov
    import synth

    torch.cuda.set_device(0)
    small = tuple(args.train_dims)
    big = tuple(args.dims) if args.dims else (32, 32, 32, 64)
    res = {}

    def prepare(dims):
        U = synth.gauge_field(dims, seed=1, s=0.5, ape_steps=3)
        ctx = ov.Context(dims, BC)
        ctx.set_gauge(torch.from_numpy(U).cuda())
        ctx.set_option("hi_prec", ov.PREC[args.hi_prec])
        ctx.set_option("chiral", int(args.chiral))
        ctx.set_sign_poly(RHO, 0.05, args.degree, 0.0)
        lmax = ctx.get_sign_poly()["lambda_max"]
        eps = 0.05
        if args.nev > 0:
            ctx.deflate(0, args.nev, args.eig_tol)
            vals, _ = ctx.get_eigenpairs(0)
            eps = (0.99 * np.abs(vals).max() / lmax) ** 2
        sign_for_delta(ctx, eps, lmax, args.sign_delta, args.degree)
        if args.nev_cg > 0:
            ctx.set_option("filter_dd", args.filter_dd)
            ctx.deflate(1, args.nev_cg, args.eig_tol)
        return ctx

    t0 = time.perf_counter()
    cs = prepare(small)
    loss = cs.net_train(nsolves=args.train_solves, steps=args.train_steps, lr=args.lr, mass=args.mass)
    curve = cs.net_loss_history()
    res["train"] = {"seconds": round(time.perf_counter() - t0, 1), "pairs": cs.net_pairs(), "loss_per_pair": loss,
                    "loss_curve": {str(i): round(float(curve[i]), 5)
                                   for i in sorted(set(list(range(0, len(curve), max(1, len(curve) // 20)))
                                                       + [len(curve) - 1]))}}
    w = cs.net_weights()
    cs.close()
    cb = prepare(big)
    cb.net_set_weights(w)
    b = torch.from_numpy(synth.point_sources(big)).cuda()
    for name, pc in (("plain", 0), ("learned", 1)):
        x = torch.empty_like(b)
        info = cb.cg_solve(b, x, mass=args.mass, tol=1e-10, max_iter=args.max_iter, precond=pc, inner_prec="f32",
                           check=False)
        res[name] = {"seconds": round(info["seconds"], 2), "iterations": info["iterations"],
                     "fallback": info["fallback"], "max_true_residual": max(info["true_residual"]),
                     "status": info["status"]}
    print(json.dumps({
        "metric": "time to 1e-10, learned flexible CG vs plain deflated CG", "value": res["learned"]["seconds"],
        "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": 1e3 * res["learned"]["seconds"],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32 + f64", "data": "synthetic",
        "config": {"workload": f"train {small}, apply {big}, 12 point sources, mass {args.mass}",
                   "hi_prec": args.hi_prec, "chiral": bool(args.chiral)}, "results": res}))


def run_peaks(args):
    """FMA throughput of this GPU (FP64 and FP32) by the library's own kernel, and the copy
    bandwidth the driver measured: the denominators of every roofline in the default line."""
    import torch

    import paper_1106_4964_gb300 as ov

    torch.cuda.set_device(0)
    hbm, kind = peaks()
    res = {p: [round(ov.measure_fma_peak(p), 1) for _ in range(3)] for p in ("f64", "f32")}
    print(json.dumps({"metric": "FMA throughput", "value": max(res["f64"]), "unit": "GFLOP/s", "n_gpus": 1,
                      "dtype": "f64", "fma_gflops": res, "hbm_gbs": hbm, "hbm_kind": kind,
                      "nominal": {"f64_gflops": FP64_NOMINAL_GFLOPS}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--inner", type=int, default=1, help="launches per step")
    ap.add_argument("--quick", action="store_true", help="headline only")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-prop", action="store_true", help="skip the propagator record of the default run")
    ap.add_argument("--prec", default=HEADLINE_PREC, choices=list(REAL_BYTES),
                    help="precision of the timed launch (profiling runs; the headline is f64)")
    ap.add_argument("--nrhs", type=int, default=1, help="right-hand sides of the timed launch (profiling runs)")
    ap.add_argument("--prop-dims", type=int, nargs=4, default=[8, 8, 8, 16])
    ap.add_argument("--prop-nev", type=int, default=16)
    ap.add_argument("--prop-mass", type=float, default=0.05)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--shape", type=int, nargs=3, default=None, metavar=("BX", "BY", "VARIANT"),
                    help="fixed dslash launch configuration instead of the autotuner (profiling)")
    ap.add_argument("--workload", default="dslash",
                    choices=["dslash", "overlap", "propagator", "learned", "project", "peaks"])
    ap.add_argument("--dims", type=int, nargs=4, default=None)
    ap.add_argument("--train-dims", type=int, nargs=4, default=[16, 16, 16, 32])
    ap.add_argument("--degree", type=int, default=200)
    ap.add_argument("--sign-delta", type=float, default=1e-10,
                    help="propagator / learned: lowest Chebyshev degree with this accuracy delta (0: --degree)")
    ap.add_argument("--nev", type=int, default=100)
    ap.add_argument("--nev-cg", type=int, default=100)
    ap.add_argument("--filter-dd", type=int, default=8)
    ap.add_argument("--eig-tol", type=float, default=1e-6)
    ap.add_argument("--mass", type=float, default=0.0)
    ap.add_argument("--delta", type=float, default=0.1)
    ap.add_argument("--cg-inner", default="f32", help="inner precisions of the propagator CG, comma separated")
    ap.add_argument("--plain-rhs", type=int, default=1,
                    help="propagator: also solve this many sources with the plain FP64 method (0: skip)")
    ap.add_argument("--chiral", type=int, default=1, choices=[0, 1],
                    help="propagator CG and D^dag D deflation on chiral sectors (one sign per application)")
    ap.add_argument("--hi-prec", default="df64", choices=["f64", "df64"],
                    help="accurate arithmetic of the propagator CG (true residuals): FP64 or double-float")
    ap.add_argument("--max-iter", type=int, default=3000)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--f64-r12", action="store_true")
    ap.add_argument("--train-solves", type=int, default=4)
    ap.add_argument("--train-steps", type=int, default=100)
    ap.add_argument("--lr", type=float, default=5e-3)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "overlap":
        run_overlap(args)
    elif args.workload == "propagator":
        run_propagator(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "project":
        run_project(args)
    elif args.workload == "peaks":
        run_peaks(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
