#!/usr/bin/env python3
"""Benchmark of the DDA hot path on GB300.

One step = the whole hot path over one batch of synthetic input: incident
field, BiCGstab solve to the relative residual 1e-5 (FP32 FFT-convolution
matvec with FP64 refinement, the production mode), and the Q_ext/Q_abs/Q_sca
reductions, for every right-hand side of the workload.

Default workload: the 64^3 sphere (137376 dipoles, m = 1.5+0.02i, x = 5,
k along x, 2 polarizations) on one GPU.  Metric: A.P matvecs per second
(right-hand-side matvecs, every precision counted) with time-to-solution,
FP32-refined vs plain FP64 on the same GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Multi-GPU (torchrun, one rank per GPU): the orientation sweep holds the
workload's right-hand sides once per rank and is sharded into contiguous RHS
blocks (paper_1202_3424_gb300.sweep), one per rank, solved with no exchange;
scaling is weak and the value is the sum over ranks.
The reference arm (--impl reference) times the CPU oracle's pairwise
O(N^2) FP64 matvec on the host cores on a bounded row sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from dda_inputs import workload  # noqa: E402

METRIC = "A.P matvecs/s (RHS x matvec per second) at tol 1e-5, FP32-refined vs FP64, time-to-solution"
UNIT = "matvec/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="sphere64")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--fp64-sequential", action="store_true",
                    help="FP64 leg solves the RHS one at a time (orientation-sweep comparison)")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the 128-RHS ellipsoid sweep block of the default solve run")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the FP64 reference solve (tol 1e-10) behind q_relerr_vs_fp64")
    ap.add_argument("--ext", type=float, default=0.5, help="nearfield mode: extension fraction on every side")
    ap.add_argument("--eta", type=float, default=0.5, help="farfield mode: ETASCA of the scattering directions")
    ap.add_argument("--mode", default="solve", choices=["solve", "matvec", "grad", "nearfield", "farfield"],
                    help="matvec: only time dda_matvec_device (for profiler captures)")
    ap.add_argument("--rhs", type=int, default=0, help="matvec mode: RHS per product (0 = workload's)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"], help="matvec mode precision")
    ap.add_argument("--cufft", action="store_true",
                    help="matvec mode: also time the same-size FFT convolution written with torch.fft (cuFFT)")
    ap.add_argument("--aniso", action="store_true",
                    help="solve/matvec modes: anisotropic version of the workload's materials (principal indices "
                         "m x (1, 1.05, 0.95), dielectric frame rotated by (0.4, 1.1, -0.6) rad)")
    ap.add_argument("--solver", default="bicgstab", choices=["bicgstab", "bicgstab2", "qmr"],
                    help="solve mode: BiCGstab (default), BiCGstab(2) (the guide's PBCGS2) or QMR for complex "
                         "symmetric A (the guide's QMRCCG)")
    ap.add_argument("--xpass", type=int, default=-1, choices=[-1, 0, 1, 2, 3],
                    help="complex64 x-pass schedule: -1 autotuned (default), 0 rows staged through shared memory, "
                         "1 + V warp-local rows with radix plan V (the last V of 64, 128, 256 and 512 points "
                         "exchanges by warp shuffles)")
    ap.add_argument("--xinv", type=int, default=None, choices=[-1, 0, 1, 2, 3],
                    help="x-inverse schedule (overrides --xpass for the inverse pass only)")
    ap.add_argument("--ypass", type=int, default=-1, choices=[-1, 0, 1],
                    help="complex64 y-pass radix plan: -1 autotuned (default), 0 or 1")
    ap.add_argument("--zpass", type=int, default=-1, choices=[-1, 0, 1, 2, 3, 4],
                    help="complex64 z-pass schedule: -1 autotuned (default), 0 component groups, "
                         "1 register-resident, 2 register-resident with octant columns, 3 and 4 as 1 and 2 "
                         "with the radix-16 plan "
                         "(forcing one makes profiler runs reproduce the tuned choice)")
    return ap.parse_args()


# ------------------------------------------------------------ distributed --
def dist_init(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("DDA_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
        return rank, world, dist
    return 0, 1, None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x, device=None):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, x, device=None):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
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
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------- algorithmic traffic ----
def target_info(ctx, w):
    """The context's target description plus the number of x rows (z, y)
    that hold at least one site."""
    info = dict(ctx.info())
    info["xrows"] = int(np.count_nonzero(np.asarray(w.grid).any(axis=2)))
    return info


def pass_bytes(kind, info, R, ncomp_tables=1):
    """Algorithmic bytes of one launch of a matvec pass over R right-hand sides:
    the data the pass must read and write once (compact vectors, padded
    intermediates, index map, Green-tensor octant)."""
    s = 8 if kind.endswith("c64") else 16
    Lx, Ly, Lz = info["Lx"], info["Ly"], info["Lz"]
    nx, ny, nz = Lx // 2, Ly // 2, Lz // 2          # lattice as the kernels see it (vacuum-padded to L/2)
    N, M = info["ndipoles"], nx * ny * nz
    u1 = 3 * nz * ny * Lx * s            # per RHS
    u2 = 3 * nz * Ly * Lx * s
    vec = 3 * N * s
    oct_ = 6 * (Lx // 2 + 1) * (Ly // 2 + 1) * (Lz // 2 + 1) * s
    if kind.startswith("xy_fwd"):             # fused x+y slice pass: P in, U2 out
        return R * (vec + u2) + 4 * M
    if kind.startswith("yx_inv"):             # fused y+x slice pass: U2 and X in, Y out
        return R * (u2 + 2 * vec) + 4 * M + N
    if kind.startswith("x_fwd"):
        return R * (vec + u1) + 4 * M
    if kind.startswith("y_fwd") or kind.startswith("y_inv"):
        return R * (u1 + u2)
    if kind.startswith("z_conv"):
        return R * 2 * u2 + oct_
    if kind.startswith("x_inv"):
        # only the x rows holding sites are read and transformed (a row
        # without sites has no output)
        rows = info.get("xrows", ny * nz)
        return R * (3 * rows * Lx * s + 2 * vec) + 4 * rows * nx + N
    return None


def pass_flops(kind, info, R):
    """Algorithmic flops (5 L log2 L per complex FFT of length L, 66 per point
    for the symmetric 3x3 complex product) of one launch over R RHS."""
    Lx, Ly, Lz = info["Lx"], info["Ly"], info["Lz"]
    nx, ny, nz = Lx // 2, Ly // 2, Lz // 2
    f = lambda L: 5 * L * math.log2(L)  # noqa: E731
    if kind.startswith("xy_fwd") or kind.startswith("yx_inv"):
        return R * 3 * (ny * nz * f(Lx) + nz * Lx * f(Ly))
    if kind.startswith("x_fwd") or kind.startswith("x_inv"):
        return R * 3 * ny * nz * f(Lx)
    if kind.startswith("y_fwd") or kind.startswith("y_inv"):
        return R * 3 * nz * Lx * f(Ly)
    if kind.startswith("z_conv"):
        return R * (2 * 3 * Lx * Ly * f(Lz) + 66 * Lx * Ly * Lz)
    return None


KERNEL_SOURCES = ["paper_1202_3424_gb300/csrc/matvec_impl.cuh", "paper_1202_3424_gb300/csrc/matvec_f32.cu",
                  "paper_1202_3424_gb300/csrc/fft.cuh", "paper_1202_3424_gb300/csrc/krylov_dev.cuh",
                  "paper_1202_3424_gb300/csrc/common.cuh", "paper_1202_3424_gb300/csrc/xwarp.cuh"]
# (pass, workload, RHS per launch) -> (summary file, kernel heading in it)
CAPTURES = {("z_conv_c64", "sphere64", 2): ("profiles/zoct16_f32_sphere64.md", "k_zconv_oct<float, 128, 2, 1>"),
            ("z_conv_c64", "ellipsoid96x64x32", 32): ("profiles/passes_f32_ellipsoid96x64x32.md",
                                                      "k_zconv_reg<float, 64, 8, 0>")}


def captured_traffic(kernel, workload_name, rhs_per_launch):
    """DRAM bytes per launch from the committed ncu summary of this kernel and
    workload, or None when there is none or the kernel source has changed
    since the capture (the summary records a hash of the sources)."""
    import hashlib
    entry = CAPTURES.get((kernel, workload_name, int(round(rhs_per_launch))))
    if entry is None or not os.path.exists(os.path.join(ROOT, entry[0])):
        return None
    path, heading = entry
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        fp = os.path.join(ROOT, f)
        if not os.path.exists(fp):
            return None
        with open(fp, "rb") as fh:
            h.update(fh.read())
    sha, traffic, in_section = None, None, False
    for line in open(os.path.join(ROOT, path)):
        if line.startswith("source_sha256:"):
            sha = line.split()[1]
        if line.startswith("### "):
            in_section = line[4:].startswith(heading)
        if in_section and line.startswith("traffic_bytes_per_launch:") and traffic is None:
            traffic = int(line.split()[1])
    return traffic if sha is not None and h.hexdigest().startswith(sha) else None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# FP64 CUDA-core peak of GB300: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz
# (derivation and the microbenchmark behind it are in the design notes).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


# ------------------------------------------------------------- gb300 arm ----
def run_gb300(args):
    import torch
    import paper_1202_3424_gb300 as dda

    rank, world, dist = dist_init(args.gpus)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args.workload)
    # weak scaling: the orientation sweep holds the workload's RHS once per
    # rank, and each rank solves its contiguous block (sweep.shard_rhs) with no
    # exchange; the per-RHS results are gathered once after the timed region
    from paper_1202_3424_gb300 import sweep
    k_all, e_all = np.tile(w.khat, (world, 1)), np.tile(w.ehat, (world, 1))
    mine = sweep.shard_rhs(len(k_all), rank, world)
    k_loc, e_loc = k_all[mine.start:mine.stop], e_all[mine.start:mine.stop]
    R = len(k_loc)
    ctx = dda.Context(local)
    stream = torch.cuda.current_stream(dev)
    dda.dda_set_stream(ctx.handle, stream.cuda_stream)
    ctx.set_target(w.grid)
    set_materials(ctx, w, args.aniso)
    t0 = time.perf_counter()
    ctx.prepare_size_parameter(w.x, dda.Precision.FP32_REFINED)
    prepare_ms = (time.perf_counter() - t0) * 1e3
    ctx.set_schedule(args.zpass)
    ctx.set_xpass((args.xpass, args.xpass if args.xinv is None else args.xinv))
    ctx.set_ypass(args.ypass)
    info = target_info(ctx, w)
    N = info["ndipoles"]
    P_dev = torch.empty((R, 3, N), dtype=torch.complex128, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2

    def step(prec, tol=1e-5):
        res, st = dda.dda_solve_device(ctx.handle, prec, k_loc, e_loc, P_dev, tol=tol, maxit=2000,
                                       solver=args.solver)
        if st != 0:
            raise RuntimeError(f"solve failed: {[r['status_name'] for r in res]}")
        return res

    def timed(prec, steps, trace=False):
        mv = 0
        per = []
        last = None
        if trace:
            dda.load_library().dda_profile_enable(ctx.handle, 1)
        barrier(dist)
        torch.cuda.synchronize()
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            last = step(prec)
            e1.record(stream)
            e1.synchronize()
            per.append(e0.elapsed_time(e1))
            mv += sum(r["matvecs"] for r in last)
        torch.cuda.synchronize()
        barrier(dist)
        stats = None
        if trace:
            stats = read_profile(dda, ctx)
            dda.load_library().dda_profile_enable(ctx.handle, 0)
        return per, mv, last, stats

    # warm-up, then the timed K steps (FP32-refined, the production mode)
    for _ in range(max(3, args.warmup)):
        step(dda.Precision.FP32_REFINED)
    clk = ClockSampler(local)
    clk.start()
    per, mv, res, _ = timed(dda.Precision.FP32_REFINED, args.steps)
    clocks = clk.stop()
    t_local = sum(per)
    t_max = max_over_ranks(dist, t_local, dev)
    mv_all = sum_over_ranks(dist, mv, dev)
    value = mv_all / (t_max / 1e3)
    ms_per_step = t_max / args.steps

    # the same steps with launch tracing: per-kernel durations for the roofline
    per_tr, mv_tr, _, kstats = timed(dda.Precision.FP32_REFINED, args.steps, trace=True)

    # plain FP64 on the same GPU (same workload, one RHS batch per step)
    fp64 = None
    if args.fp64_steps > 0 and not args.fp64_sequential:
        step(dda.Precision.FP64)
        per64, mv64, res64, _ = timed(dda.Precision.FP64, args.fp64_steps)
        fp64 = {"time_to_solution_ms": sum(per64) / len(per64), "matvecs_per_s": mv64 / (sum(per64) / 1e3),
                "iters": [r["iters"] for r in res64], "resid_rel": [r["resid_rel"] for r in res64],
                "q": [[r["qext"], r["qabs"], r["qsca"]] for r in res64]}
    elif args.fp64_steps > 0:
        # orientation sweep as a plain FP64 single-RHS loop: one solve per RHS
        P1 = torch.empty((1, 3, N), dtype=torch.complex128, device=dev)
        dda.dda_solve_device(ctx.handle, dda.Precision.FP64, k_loc[:1], e_loc[:1], P1, tol=1e-5, maxit=2000)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        mv64 = 0
        it64 = []
        for r_ in range(R):
            rr, st = dda.dda_solve_device(ctx.handle, dda.Precision.FP64, k_loc[r_:r_ + 1], e_loc[r_:r_ + 1], P1,
                                          tol=1e-5, maxit=2000)
            mv64 += rr[0]["matvecs"]
            it64.append(rr[0]["iters"])
        e1.record(stream)
        e1.synchronize()
        t64 = e0.elapsed_time(e1)
        fp64 = {"time_to_solution_ms": t64, "matvecs_per_s": mv64 / (t64 / 1e3), "mode": "sequential single-RHS",
                "iters_mean": sum(it64) / len(it64)}

    # end to end through the host-buffer C-ABI call (P copied back every step)
    e2e = None
    if not args.no_e2e:
        k = np.ascontiguousarray(k_loc)
        e = np.ascontiguousarray(e_loc)
        ctx.solve(dda.Precision.FP32_REFINED, k, e, tol=1e-5, maxit=2000, solver=args.solver)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mv_e2e = 0
        for _ in range(args.steps):
            r_e2e, P_host, st = ctx.solve(dda.Precision.FP32_REFINED, k, e, tol=1e-5, maxit=2000, solver=args.solver)
            mv_e2e += sum(r["matvecs"] for r in r_e2e)
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(dist, time.perf_counter() - t0, dev)
        e2e = {"value": sum_over_ranks(dist, mv_e2e, dev) / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(k.nbytes + e.nbytes), "d2h_bytes_per_step": int(P_host.nbytes + 72 * R),
               "time_to_solution_ms": t_e2e * 1e3 / args.steps}

    # the matvec schedules the autotuner chose for this RHS count (cached by now)
    schedule = {"solve": ctx.get_solve_schedule(R),
                "plain_matvec": {"zpass": ctx.get_schedule(R), "xpass_fwd_inv": list(ctx.get_xpass(R)),
                                 "ypass": ctx.get_ypass(R)}}
    roof = roofline(kstats, info, R, w.name)
    # complex64 RHS-matvecs per traced step: 2 per BiCGstab (4 per BiCGstab(2)) iteration of every RHS
    per_iter = {"bicgstab": 2, "bicgstab2": 4, "qmr": 1}[args.solver]
    mv_roof = matvec_roofline(kstats, info, "c64",
                              rhs_matvecs=len(per_tr) * sum(per_iter * r["iters"] for r in res),
                              fused_vectors=FUSED_VECTORS_PER_MATVEC.get(args.solver, 0.0)) \
        if kstats else None
    launches = int(sum(s["launches"] for s in kstats.values()) / args.steps) * args.steps if kstats else 0

    # every rank's per-RHS results, in sweep order (the sweep's one collective)
    def solve_block(kb, eb):
        rr, _ = dda.dda_solve_device(ctx.handle, dda.Precision.FP32_REFINED, kb, eb, P_dev[:len(kb)], tol=1e-5,
                                     maxit=2000, solver=args.solver)
        return [[r["qext"], r["qabs"], r["qsca"], r["resid_rel"]] for r in rr]
    swept = sweep.solve_sweep(solve_block, k_all, e_all, dist)

    # error of the production mode per result, against an FP64 solve to 1e-10
    accuracy = None
    if not args.no_accuracy:
        accuracy = accuracy_vs_fp64(dda, ctx, k_loc, e_loc, P_dev, res, fp64["q"] if fp64 and "q" in fp64 else None)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, info, budget_s=12.0)

    ell_sweep = None
    if args.mode == "solve" and args.workload == "sphere64" and not args.no_sweep and not args.aniso \
            and args.solver == "bicgstab" and world == 1:
        ctx.close()
        ctx = None
        ell_sweep = ellipsoid_sweep(dda, dev, stream, flush, dist)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64 matvec / f64 refinement", "data": "synthetic",
            "config": {"workload": f"{w.name}: lattice {info['nx']}x{info['ny']}x{info['nz']}, N={N} dipoles, "
                                   f"{materials_note(w, args.aniso)}, x={w.x}, {R} RHS, tol 1e-5, "
                                   f"{ {'bicgstab': 'BiCGstab', 'bicgstab2': 'BiCGstab(2)', 'qmr': 'QMR'}[args.solver]}",
                       "global_batch": len(k_all), "padded_grid": [info["Lx"], info["Ly"], info["Lz"]],
                       "parallelism": f"rhs-sharded x{world} (sweep.shard_rhs blocks, no exchange; results "
                                      f"gathered after timing)", "l2": "256 MB buffer written between steps"},
            "time_to_solution_ms": ms_per_step,
            "iters": [r["iters"] for r in res], "outer_iters": [r["outer_iters"] for r in res],
            "matvecs_per_step": mv / args.steps, "resid_rel": [r["resid_rel"] for r in res],
            "q": [r[:3] for r in swept], "sweep_rhs": len(swept),
            "fp64_plain": fp64, "speedup_vs_fp64": fp64["time_to_solution_ms"] / ms_per_step if fp64 else None,
            "prepare_ms": prepare_ms,
            "traced_ms_per_step": sum(per_tr) / len(per_tr),
            "kernels": {k_: {"launches": v["launches"], "ms": v["ms"], "share": v["share"]} for k_, v in kstats.items()},
            "roofline": roof, "matvec_roofline": mv_roof, "schedule": schedule,
            "q_relerr_vs_fp64": accuracy,
            "ellipsoid_sweep_128rhs": ell_sweep,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if ctx is not None:
        ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def _q_relerr(q, qref):
    """Per RHS: |Q - Q_ref| / |Q_ref| for Q_ext, Q_abs, Q_sca."""
    return [[abs(a - b) / abs(b) for a, b in zip(qi, qr)] for qi, qr in zip(q, qref)]


def accuracy_vs_fp64(dda, ctx, khat, ehat, P_dev, res, q_fp64_tol5=None, tol_ref=1e-10):
    """Error of the FP32-refined results (tol 1e-5) per RHS and per
    efficiency factor, against a plain FP64 solve of the same RHS to
    tol_ref on the same GPU (the FP64 path matches the CPU oracle to 1e-10).
    The FP64 solve to 1e-5 is shown beside it: both stop at the same
    residual, so their distance from the tight solution is of one size."""
    import torch
    Pref = torch.empty_like(P_dev)
    rref, st = dda.dda_solve_device(ctx.handle, dda.Precision.FP64, khat, ehat, Pref, tol=tol_ref, maxit=4000)
    if st != 0:
        return {"error": f"FP64 reference solve status {st}"}
    qref = [[r["qext"], r["qabs"], r["qsca"]] for r in rref]
    q = [[r["qext"], r["qabs"], r["qsca"]] for r in res]
    err = _q_relerr(q, qref)
    out = {"what": "per RHS [Q_ext, Q_abs, Q_sca] relative error of the FP32-refined solve (tol 1e-5) vs a "
                   f"plain FP64 solve to tol {tol_ref:g}",
           "fp32_refined": err, "max": max(max(e) for e in err), "q_ref": qref,
           "ref_resid_rel": [r["resid_rel"] for r in rref]}
    if q_fp64_tol5 is not None:
        e64 = _q_relerr(q_fp64_tol5, qref)
        out["fp64_tol1e-5"] = e64
        out["fp64_tol1e-5_max"] = max(max(e) for e in e64)
    return out


def ellipsoid_sweep(dda, dev, stream, flush, dist, steps=3, warmup=2):
    """The 128-RHS orientation sweep of the 3:2:1 ellipsoid (96x64x32, 64
    seeded directions x 2 polarizations): one batched FP32-refined solve of
    all RHS (shared Green tensor, per-RHS masks, graph replay) against 128
    sequential single-RHS plain FP64 solves, the whole matvec alone and
    inside the solve against HBM, and the per-result error on 16 RHS."""
    import torch
    w = workload("ellipsoid96x64x32")
    R = w.nrhs
    ctx = dda.Context(dev.index)
    dda.dda_set_stream(ctx.handle, stream.cuda_stream)
    ctx.set_target(w.grid)
    ctx.set_materials(w.m)
    ctx.prepare_size_parameter(w.x, dda.Precision.FP32_REFINED)
    info = target_info(ctx, w)
    N = info["ndipoles"]
    P = torch.empty((R, 3, N), dtype=torch.complex128, device=dev)

    def solve(prec, k, e, out, tol=1e-5):
        rr, st = dda.dda_solve_device(ctx.handle, prec, k, e, out, tol=tol, maxit=3000)
        if st != 0:
            raise RuntimeError(f"sweep solve failed: {[r['status_name'] for r in rr]}")
        return rr

    def event_ms(fn):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), out

    for _ in range(warmup):
        solve(dda.Precision.FP32_REFINED, w.khat, w.ehat, P)
    torch.cuda.synchronize()
    per, res = [], None
    for _ in range(steps):
        ms, res = event_ms(lambda: solve(dda.Precision.FP32_REFINED, w.khat, w.ehat, P))
        per.append(ms)
    t_b = statistics.median(per)
    mv = sum(r["matvecs"] for r in res)
    # traced solve: the five passes inside the solve against HBM
    L = dda.load_library()
    L.dda_profile_enable(ctx.handle, 1)
    solve(dda.Precision.FP32_REFINED, w.khat, w.ehat, P)
    kin = read_profile(dda, ctx)
    L.dda_profile_enable(ctx.handle, 0)
    mv_in = matvec_roofline(kin, info, "c64", rhs_matvecs=sum(2 * r["iters"] for r in res),
                            fused_vectors=FUSED_VECTORS_PER_MATVEC["bicgstab"])
    # the matvec alone (128 RHS per product)
    x = torch.randn((R, 3, N), dtype=torch.complex64, device=dev, generator=torch.Generator(device=dev).manual_seed(1))
    y = torch.empty_like(x)
    for _ in range(3):
        dda.dda_matvec_device(ctx.handle, 2, w.khat, w.ehat, x, y)
    ms_mv, _ = event_ms(lambda: [dda.dda_matvec_device(ctx.handle, 2, w.khat, w.ehat, x, y) for _ in range(10)])
    L.dda_profile_enable(ctx.handle, 1)
    for _ in range(10):
        dda.dda_matvec_device(ctx.handle, 2, w.khat, w.ehat, x, y)
    kmv = read_profile(dda, ctx)
    L.dda_profile_enable(ctx.handle, 0)
    mv_alone = matvec_roofline(kmv, info, "c64")
    del x, y
    # 128 sequential single-RHS plain FP64 solves (the orientation loop without batching)
    P1 = torch.empty((1, 3, N), dtype=torch.complex128, device=dev)
    solve(dda.Precision.FP64, w.khat[:1], w.ehat[:1], P1)
    torch.cuda.synchronize()
    t_64, seq = event_ms(lambda: [solve(dda.Precision.FP64, w.khat[i:i + 1], w.ehat[i:i + 1], P1)[0]
                                  for i in range(R)])
    # per-result error on the first 16 RHS against FP64 to 1e-10
    n_acc = 16
    P16 = torch.empty((n_acc, 3, N), dtype=torch.complex128, device=dev)
    rref = solve(dda.Precision.FP64, w.khat[:n_acc], w.ehat[:n_acc], P16, tol=1e-10)
    err = _q_relerr([[r["qext"], r["qabs"], r["qsca"]] for r in res[:n_acc]],
                    [[r["qext"], r["qabs"], r["qsca"]] for r in rref])
    err64 = _q_relerr([[r["qext"], r["qabs"], r["qsca"]] for r in seq[:n_acc]],
                      [[r["qext"], r["qabs"], r["qsca"]] for r in rref])
    ctx.close()
    return {"workload": f"{w.name}: lattice {info['nx']}x{info['ny']}x{info['nz']}, N={N}, m={w.m}, x={w.x}, "
                        f"{R} RHS (64 seeded directions x 2 polarizations), tol 1e-5",
            "batched_fp32_refined_ms": t_b, "batched_rhs_matvecs_per_s": mv / (t_b / 1e3),
            "iters_min_max": [min(r["iters"] for r in res), max(r["iters"] for r in res)],
            "max_resid_rel": max(r["resid_rel"] for r in res),
            "sequential_fp64_single_rhs_ms": t_64, "speedup_vs_sequential_fp64": t_64 / t_b,
            "matvec_alone_ms": ms_mv / 10, "matvec_alone_roofline": mv_alone, "matvec_in_solve_roofline": mv_in,
            "q_relerr_vs_fp64_first16": {"fp32_refined": err, "max": max(max(e) for e in err),
                                         "fp64_tol1e-5_max": max(max(e) for e in err64),
                                         "ref": "plain FP64 solve to tol 1e-10"},
            "steps": steps, "warmup": warmup, "l2": "256 MB buffer written before each timed solve"}


def read_profile(dda, ctx):
    import ctypes

    class Stat(ctypes.Structure):
        _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                    ("units", ctypes.c_double)]

    lib = dda.load_library()
    lib.dda_profile_read.argtypes = [ctypes.c_void_p, ctypes.POINTER(Stat), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    arr = (Stat * 64)()
    n = ctypes.c_int()
    lib.dda_profile_read(ctx.handle, arr, 64, ctypes.byref(n))
    out = {}
    total = sum(arr[i].total_ms for i in range(n.value))
    for i in range(n.value):
        out[arr[i].name.decode()] = {"launches": arr[i].launches, "ms": arr[i].total_ms, "units": arr[i].units,
                                     "share": arr[i].total_ms / total if total else 0.0}
    return out


def roofline(kstats, info, R, workload_name=None):
    if not kstats:
        return None
    hbm, src = load_peaks()
    # dominant kernel among the matvec passes (the hot path's bulk)
    cands = {k: v for k, v in kstats.items() if pass_bytes(k, info, 1) is not None}
    name = max(cands, key=lambda k: cands[k]["ms"])
    v = cands[name]
    avg_ms = v["ms"] / v["launches"]
    units_per_launch = v["units"] / v["launches"]
    if name.endswith("c128"):
        fl = pass_flops(name, info, units_per_launch)
        ach = fl / (avg_ms / 1e3) / 1e12
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": None, "avg_launch_ms": avg_ms,
                "rhs_per_launch": units_per_launch, "peak_source": "derived FP64 (152 SM x 2 DFMA/clk x 2.07 GHz)"}
    b = pass_bytes(name, info, units_per_launch)
    ach = b / (avg_ms / 1e3) / 1e9
    traffic = captured_traffic(name, workload_name, units_per_launch)
    return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": traffic, "traffic_note": "ncu cold-cache DRAM bytes per launch (profiles/)" if traffic else None,
            "avg_launch_ms": avg_ms, "algorithmic_bytes_per_launch": b,
            "rhs_per_launch": units_per_launch, "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"}


# Vector traffic the BiCGstab updates fused into the x passes add per
# RHS-matvec, in units of one compact vector (3N complex): over the two
# matvecs of an iteration, the first gather reads s, t, p, v, x and writes r,
# x, p (7 more than a plain gather of p), the second gather reads r, v and
# writes s (2 more), and each scatter reads rhat (2 more): 11 per iteration,
# 5.5 per matvec.  (The iteration has no other kernel.)
FUSED_VECTORS_PER_MATVEC = {"bicgstab": 5.5}


def matvec_roofline(kstats, info, suffix="c64", rhs_matvecs=None, fused_vectors=0.0):
    """The whole FFT-convolution matvec (its five passes together) against
    HBM: algorithmic bytes of all launches of the passes / their total time.

    Bytes per launch are pass_bytes (compact vectors of N sites, padded
    intermediates, index maps, Green octant).  The profiler's units count
    the RHS a launch was given; inside a solve RHS that have converged are
    skipped, so rhs_matvecs (the RHS-matvecs actually done, from the solver's
    iteration counts) replaces them there, and fused_vectors (compact
    vectors per RHS-matvec that the fused Krylov updates read or write in
    the x passes) adds that traffic.  `survey_model` also gives the
    lattice-wide model (81 R + 6) M s per matvec of R RHS (M = lattice
    sites, P read and written on the whole lattice)."""
    hbm, src = load_peaks()
    kinds = [k for k in kstats if k.endswith(suffix) and pass_bytes(k, info, 1) is not None]
    if len(kinds) not in (3, 5):   # fused slice passes + z, or the five separate passes
        return None
    ms = sum(kstats[k]["ms"] for k in kinds)
    b = 0.0
    for k in kinds:
        fixed = pass_bytes(k, info, 0)
        per_rhs = pass_bytes(k, info, 1) - fixed
        units = kstats[k]["units"] if rhs_matvecs is None else rhs_matvecs
        b += per_rhs * units + fixed * kstats[k]["launches"]
    s = 8 if suffix == "c64" else 16
    fused_bytes = fused_vectors * 3 * info["ndipoles"] * s * (rhs_matvecs or 0)
    b += fused_bytes
    ach = b / (ms / 1e3) / 1e9
    M = (info["Lx"] // 2) * (info["Ly"] // 2) * (info["Lz"] // 2)
    zk = [k for k in kinds if k.startswith("z_conv")][0]
    units = kstats[zk]["units"] if rhs_matvecs is None else rhs_matvecs
    sb = (81 * units + 6 * kstats[zk]["launches"]) * M * s
    sach = sb / (ms / 1e3) / 1e9
    return {"passes": sorted(kinds), "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": ach / hbm, "ms": ms, "algorithmic_bytes": b, "fused_update_bytes": fused_bytes,
            "rhs_matvecs": units,
            "survey_model": {"bytes": sb, "achieved": sach, "frac": sach / hbm},
            "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"}


# ----------------------------------------------------------- CPU baseline ----
def _oracle_rows_rate(w, budget_s, kd):
    """Rows of A.P per second of the oracle's pairwise matvec on this host."""
    from oracle import dda as odda
    from oracle import pairwise
    r, comp = odda.site_positions(w.grid)
    N = len(r)
    eps = (np.asarray(w.m) ** 2)[comp - 1]
    beta = odda.ldr_inverse_polarizability(eps, kd, w.khat[0], w.ehat[0])
    P = np.random.default_rng(1).standard_normal((N, 3)) + 0j
    rng = np.random.default_rng(2)
    nrows = 64
    t0 = time.perf_counter()
    _, nt = pairwise.matvec(r, kd, beta, P, rows=rng.choice(N, nrows, replace=False))
    dt = time.perf_counter() - t0
    nrows = max(64, int(nrows * budget_s / max(dt, 1e-6)))
    nrows = min(nrows, N)
    t0 = time.perf_counter()
    _, nt = pairwise.matvec(r, kd, beta, P, rows=rng.choice(N, nrows, replace=False))
    dt = time.perf_counter() - t0
    return nrows / dt, nrows, N, nt, dt


ANISO_FACTORS = (1.0, 1.05, 0.95)
ANISO_ANGLES = (0.4, 1.1, -0.6)


def set_materials(ctx, w, aniso):
    """The workload's materials, or (aniso) a biaxial material per composition
    with principal indices m * ANISO_FACTORS in a dielectric frame rotated by
    ANISO_ANGLES."""
    if aniso:
        ctx.set_anisotropic_materials([[m * f for f in ANISO_FACTORS] for m in w.m], [ANISO_ANGLES] * len(w.m))
    else:
        ctx.set_materials(w.m)


def materials_note(w, aniso):
    if not aniso:
        return f"m={w.m}"
    return f"anisotropic: m x {ANISO_FACTORS} along the dielectric axes, (theta,phi,beta)_DF={ANISO_ANGLES}, m={w.m}"


def cpu_baseline(w, info, budget_s=12.0):
    rate, nrows, N, nt, dt = _oracle_rows_rate(w, budget_s, info["kd"])
    return {"value": rate / N, "unit": UNIT, "cores": nt, "kind": "oracle",
            "sample": f"oracle pairwise O(N^2) FP64 matvec (C/OpenMP) on {nrows} of {N} rows of one A.P "
                      f"({dt:.1f} s), extrapolated to full RHS-matvecs per second"}


# --------------------------------------------------------- reference arm ----
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import dda as odda
    w = workload(args.workload)
    N = w.ndipoles
    kd = odda.kd_from_size_parameter(w.x, N)
    per = []
    for i in range(args.warmup + args.steps):
        rate, nrows, N, nt, dt = _oracle_rows_rate(w, 4.0, kd)
        if i >= args.warmup:
            per.append((rate, nrows, dt))
    rates = [p[0] for p in per]
    value = statistics.median(rates) / N
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median([p[2] for p in per]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"{w.name}, N={N} dipoles, {w.nrhs} RHS"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle",
                             "sample": f"per step: {per[0][1]} of {N} rows of the pairwise O(N^2) matvec, "
                                       f"extrapolated to full matvecs"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_matvec_only(args):
    """Time dda_matvec_device alone (used for profiler captures of the passes)."""
    import torch
    import paper_1202_3424_gb300 as dda
    w = workload(args.workload)
    R = args.rhs or w.nrhs
    ctx = dda.Context(0)
    ctx.set_target(w.grid)
    set_materials(ctx, w, args.aniso)
    ctx.prepare_size_parameter(w.x, dda.Precision.FP32_REFINED)
    ctx.set_schedule(args.zpass)
    ctx.set_xpass((args.xpass, args.xpass if args.xinv is None else args.xinv))
    ctx.set_ypass(args.ypass)
    N = ctx.info()["ndipoles"]
    k = np.resize(w.khat, (R, 3))
    e = np.resize(w.ehat, (R, 3))
    prec, dt = (2, torch.complex64) if args.precision == "fp32" else (0, torch.complex128)
    g = torch.Generator(device="cuda").manual_seed(1)
    x = torch.randn((R, 3, N), dtype=dt, device="cuda", generator=g)
    y = torch.empty_like(x)
    for _ in range(max(3, args.warmup)):
        dda.dda_matvec_device(ctx.handle, prec, k, e, x, y)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        dda.dda_matvec_device(ctx.handle, prec, k, e, x, y)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    L = dda.load_library()
    L.dda_profile_enable(ctx.handle, 1)
    for _ in range(args.steps):
        dda.dda_matvec_device(ctx.handle, prec, k, e, x, y)
    kst = read_profile(dda, ctx)
    L.dda_profile_enable(ctx.handle, 0)
    info = target_info(ctx, w)
    kern = {}
    for name, v in kst.items():
        avg = v["ms"] / v["launches"]
        b = pass_bytes(name, info, v["units"] / v["launches"])
        kern[name] = {"avg_ms": avg, "gbs": (b / (avg / 1e3) / 1e9) if b else None}
    mv_roof = matvec_roofline(kst, info, "c64" if args.precision == "fp32" else "c128")
    zpass = ctx.get_schedule(R) if args.precision == "fp32" else 0
    xpass = list(ctx.get_xpass(R)) if args.precision == "fp32" else 0
    ypass = ctx.get_ypass(R) if args.precision == "fp32" else 0
    line = {"mode": "matvec", "workload": w.name, "rhs": R, "precision": args.precision, "zpass": zpass,
            "xpass": xpass, "ypass": ypass,
            "ms_per_matvec": ms, "rhs_matvecs_per_s": R / (ms / 1e3), "kernels": kern, "matvec_roofline": mv_roof}
    if args.cufft:
        line["cufft_comparison"] = cufft_matvec_timing(w, info, R, dt, x, args.steps)
        line["cufft_comparison"]["speedup_of_library"] = line["cufft_comparison"]["ms_per_matvec"] / ms
    print(json.dumps(line), flush=True)
    ctx.close()


def cufft_matvec_timing(w, info, R, dt, x, steps, chunk_bytes=4 << 30):
    """Timed comparison only: the same-size FFT-convolution matvec written with
    torch.fft (cuFFT) -- scatter of the compact vectors into the zero-padded
    grid, 3-D FFTs of the three components, the symmetric 3x3 product with a
    full-grid Fourier-space tensor, inverse FFTs, gather at the occupied sites
    and the diagonal term.  The tensor and the diagonal are random (their
    values do not change the timing), so the result is not the DDA product."""
    import torch
    Lx, Ly, Lz = info["Lx"], info["Ly"], info["Lz"]
    nz, ny, nx = w.grid.shape
    dev = x.device
    sites = torch.as_tensor(np.flatnonzero(w.grid.reshape(-1) != 0), device=dev)
    iz, rem = sites // (ny * nx), sites % (ny * nx)
    iy, ix = rem // nx, rem % nx
    flat = (iz * Ly + iy) * Lx + ix                      # site -> padded-grid index
    g = torch.Generator(device="cuda").manual_seed(2)
    G = torch.randn((6, Lz, Ly, Lx), dtype=dt, device=dev, generator=g)
    beta = torch.randn((R, 1, x.shape[2]), dtype=dt, device=dev, generator=g)
    per_rhs = 3 * Lz * Ly * Lx * x.element_size()
    rc = max(1, min(R, chunk_bytes // per_rhs))
    y = torch.empty_like(x)

    def matvec():
        for r0 in range(0, R, rc):
            xs = x[r0:r0 + rc]
            n = xs.shape[0]
            pad = torch.zeros((n, 3, Lz * Ly * Lx), dtype=dt, device=dev)
            pad[:, :, flat] = xs
            f = torch.fft.fftn(pad.view(n, 3, Lz, Ly, Lx), dim=(-3, -2, -1))
            px, py, pz = f[:, 0], f[:, 1], f[:, 2]
            f = torch.stack((G[0] * px + G[1] * py + G[2] * pz, G[1] * px + G[3] * py + G[4] * pz,
                             G[2] * px + G[4] * py + G[5] * pz), dim=1)
            out = torch.fft.ifftn(f, dim=(-3, -2, -1)).view(n, 3, -1)
            y[r0:r0 + n] = out[:, :, flat] + beta[r0:r0 + n] * xs

    for _ in range(3):
        matvec()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        matvec()
    e1.record()
    e1.synchronize()
    return {"ms_per_matvec": e0.elapsed_time(e1) / steps, "rhs_per_chunk": rc,
            "what": "torch.fft (cuFFT) convolution of the same padded size, random full-grid tensor"}


def run_grad(args):
    """Time dda_grad_qabs (forward solve + adjoint solve + gradient) in FP64."""
    import torch
    import paper_1202_3424_gb300 as dda
    w = workload(args.workload)
    ctx = dda.Context(0)
    ctx.set_target(w.grid)
    ctx.set_materials(w.m)
    ctx.prepare_size_parameter(w.x, dda.Precision.FP32_REFINED)
    k, e = w.khat[:1], w.ehat[:1]
    out = {}
    for name, prec in (("fp64", dda.Precision.FP64), ("fp32_refined", dda.Precision.FP32_REFINED)):
        for _ in range(max(1, args.warmup)):
            ctx.grad_qabs(prec, k, e, tol=1e-5)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            gre, gim, P, (rf, ra) = ctx.grad_qabs(prec, k, e, tol=1e-5)
        torch.cuda.synchronize()
        out[name] = {"ms_per_gradient": (time.perf_counter() - t0) * 1e3 / args.steps,
                     "forward_iters": rf["iters"], "adjoint_iters": ra["iters"], "qabs": rf["qabs"],
                     "grad_norm": float(np.sqrt(np.sum(gre ** 2 + gim ** 2)))}
    print(json.dumps({"mode": "grad", "workload": w.name, "ndipoles": ctx.info()["ndipoles"], **out}), flush=True)
    ctx.close()


def _fft_length(n):
    """Smallest supported padded length >= 2n (the library's rule)."""
    for L in (16, 32, 48, 64, 96, 128, 192, 256, 384, 512):
        if L >= 2 * n:
            return L
    return None


def run_nearfield(args):
    """Time dda_nearfield (E_inc and E_sca on the extended box) after a solve."""
    import torch
    import paper_1202_3424_gb300 as dda
    w = workload(args.workload)
    ctx = dda.Context(0)
    ctx.set_target(w.grid)
    ctx.set_materials(w.m)
    ctx.prepare_size_parameter(w.x, dda.Precision.FP32_REFINED)
    R = args.rhs or w.nrhs
    k, e = np.resize(w.khat, (R, 3)), np.resize(w.ehat, (R, 3))
    res, P, _ = ctx.solve(dda.Precision.FP32_REFINED, k, e, tol=1e-5)
    ext = [args.ext] * 6
    dims, off = ctx.nearfield_dims(ext)
    prec = 2 if args.precision == "fp32" else 0
    out = {}
    for _ in range(max(1, args.warmup)):
        ctx.nearfield(prec, k, e, P, ext)
    torch.cuda.synchronize()
    L = dda.load_library()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Ei, Es, _, _ = ctx.nearfield(prec, k, e, P, ext)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / args.steps
    L.dda_profile_enable(ctx.handle, 1)
    ctx.nearfield(prec, k, e, P, ext)
    kst = read_profile(dda, ctx)
    L.dda_profile_enable(ctx.handle, 0)
    box = {"Lx": _fft_length(dims[0]), "Ly": _fft_length(dims[1]), "Lz": _fft_length(dims[2]),
           "ndipoles": dims[0] * dims[1] * dims[2]}
    suffix = "c64" if prec == 2 else "c128"
    ne = dims[0] * dims[1] * dims[2]
    print(json.dumps({"mode": "nearfield", "workload": w.name, "rhs": R, "precision": args.precision, "ext": ext,
                      "box": dims, "offset": off, "padded_grid": [box["Lx"], box["Ly"], box["Lz"]],
                      "ms_per_call": ms, "field_points_per_s": R * ne / (ms / 1e3),
                      "kernels": {k_: {"launches": v["launches"], "ms": v["ms"]} for k_, v in kst.items()},
                      "convolution_roofline": matvec_roofline(kst, box, suffix),
                      "max_abs_E": float(np.abs(Ei + Es).max())}), flush=True)
    ctx.close()


def run_farfield(args):
    """Time dda_angular_averages (far-field amplitudes on the guide's directions + Q_sca, g) after a solve."""
    import torch
    import paper_1202_3424_gb300 as dda
    w = workload(args.workload)
    ctx = dda.Context(0)
    ctx.set_target(w.grid)
    ctx.set_materials(w.m)
    ctx.prepare_size_parameter(w.x, dda.Precision.FP32_REFINED)
    R = args.rhs or w.nrhs
    k, e = np.resize(w.khat, (R, 3)), np.resize(w.ehat, (R, 3))
    res, P, _ = ctx.solve(dda.Precision.FP32_REFINED, k, e, tol=1e-5)
    prec = 2 if args.precision == "fp32" else 0
    for _ in range(max(1, args.warmup)):
        ctx.angular_averages(prec, k, P, eta=args.eta)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        out, nd = ctx.angular_averages(prec, k, P, eta=args.eta)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / args.steps
    L = dda.load_library()
    L.dda_profile_enable(ctx.handle, 1)
    ctx.angular_averages(prec, k, P, eta=args.eta)
    kst = read_profile(dda, ctx)
    L.dda_profile_enable(ctx.handle, 0)
    N = ctx.info()["ndipoles"]
    kern = kst.get("far_field", {"ms": 0.0, "launches": 0})
    qsolve = np.array([r["qext"] - r["qabs"] for r in res])
    print(json.dumps({"mode": "farfield", "workload": w.name, "rhs": R, "precision": args.precision, "eta": args.eta,
                      "directions": nd, "ms_per_call": ms, "kernel_ms": kern["ms"],
                      "site_direction_rhs_per_s": N * nd * R / (kern["ms"] / 1e3) if kern["ms"] else None,
                      "qsca_mean": float(out[:, 0].mean()), "qsca_solve_mean": float(qsolve.mean()),
                      "g_mean": float(out[:, 1].mean()), "cos2_mean": float(out[:, 2].mean())}), flush=True)
    ctx.close()


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.mode == "matvec":
        run_matvec_only(a)
    elif a.mode == "farfield":
        run_farfield(a)
    elif a.mode == "nearfield":
        run_nearfield(a)
    elif a.mode == "grad":
        run_grad(a)
    else:
        run_gb300(a)
