"""Benchmark of the coupled FFT-EVP / phase-field DRX hot path on GB300.

One step = one DRX increment of the 128^3 / 256-grain polycrystal: the converged Green-operator
fixed point with per-voxel Newton (evp_increment), nucleation (drx_nucleate) and five phase-field
steps (pf_step). Headline: FFT-EVP voxel-iterations/s in the FP32-mixed path; the FP64 path runs
on the same seeded input for the precision comparison (macro stress error, voxel stress error,
recrystallised fraction) and its own throughput.

  python bench.py [--gpus N --steps K --warmup W] [--impl native|reference]

Multi-GPU: the path has no exchange step (replicas only), so each rank runs an
independent replica; the value is the sum over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1509_04953_gb300 import synth  # noqa: E402

METRIC = "FFT-EVP voxel-iters/s + DRX increments/s at 128^3, FP32-mixed vs FP64 at <=1e-4"
UNIT = "voxel-iterations/s"
# algorithmic floating-point operations of the per-voxel local solve
NEWTON_FLOPS_EVAL = 1140      # one residual + tangent + potential evaluation (12 slip systems)
NEWTON_FLOPS_RESID = 544      # one residual + potential evaluation without the tangent
NEWTON_FLOPS_FACTOR = 80      # one 6x6 LDL^T factorisation
NEWTON_FLOPS_SOLVE = 72       # the two triangular solves of one Newton step
# Nominal FMA-pipe peaks (SMs x lanes x 2 x maximum SM clock for FP32; the data-sheet FP64 rate), used only if the
# library's FMA-chain measurement (evp_fma_throughput) fails; bench.py measures both in the same run.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP64_PEAK_TFLOPS = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="cu128")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "mixed_fast", "fp64"],
                    help="precision of the timed solver (the headline is the mixed path)")
    ap.add_argument("--fp64-steps", type=int, default=-1, help="FP64 comparison increments (-1 = warmup+steps)")
    ap.add_argument("--fast-steps", type=int, default=2, help="timed increments of the FP32-solve mixed path")
    ap.add_argument("--al-steps", type=int, default=1, help="run the augmented-Lagrangian companion (0 = skip)")
    ap.add_argument("--pf2-steps", type=int, default=2,
                    help="timed increments of the companion on the 2:1 phase-field grid (0 = skip)")
    ap.add_argument("--mr-steps", type=int, default=2,
                    help="timed increments of the Ma-Roters companion (the paper's dislocation law; 0 = skip)")
    ap.add_argument("--mr-fp64-steps", type=int, default=2, help="FP64 Ma-Roters comparison increments (0 = skip)")
    ap.add_argument("--fft-reps", type=int, default=20,
                    help="repetitions of the FFT comparison against cuFFT (torch.fft; 0 = skip)")
    ap.add_argument("--trajectory", type=int, default=500,
                    help="increments of the full-run mixed vs FP64 comparison and DRX window (0 = skip)")
    ap.add_argument("--trajectory-fp64-scheme", default="al", choices=["basic", "al"],
                    help="fixed-point scheme of the FP64 reference run (both reach the same solution)")
    ap.add_argument("--drx-window", type=int, default=10, help="timed increments of the DRX-regime window")
    ap.add_argument("--large-steps", type=int, default=3,
                    help="timed DRX increments of the 256^3 / 1024-grain companion (0 = skip it)")
    ap.add_argument("--large-adjoint", type=int, default=16,
                    help="increments of the 256^3 checkpointed adjoint sweep (0 = skip)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tol", type=float, default=1e-6, help="fixed-point tolerance of the mixed path")
    ap.add_argument("--ref-scale", type=float, default=1.0,
                    help="basic scheme: reference shear modulus mu_Voigt / ref_scale (1 = Voigt); same solution")
    ap.add_argument("--soft-ref-steps", type=int, default=2,
                    help="timed increments of the companion with the softer reference medium (0 = skip)")
    ap.add_argument("--soft-ref", type=float, default=1.3, help="its ref_scale")
    ap.add_argument("--tol64", type=float, default=1e-8, help="fixed-point tolerance of the FP64 path")
    ap.add_argument("--newton-tol", type=float, default=None,
                    help="local-solve tolerance (default: the library's per precision)")
    ap.add_argument("--newton-adapt", type=float, default=None,
                    help="adaptive local tolerance factor of the basic scheme (default: the library's per precision)")
    return ap.parse_args()


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "power_w_max": max(power),
                "samples": len(sm), "reasons": sorted(reasons)}


def workload_inputs(wl):
    seeds = synth.voronoi_seeds(wl.n, wl.grains, wl.seed)
    quat = synth.orientations(wl.grains, wl.seed)
    return seeds, quat


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------------------------
def run_steps(solver, steps, dE33, dt, pf_steps, torch, record=None):
    """Run `steps` DRX increments; returns per-step (evp_ms, step_ms, iterations, stats)."""
    out = []
    st = solver.stream
    for s in range(steps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(st)
        rc, es = solver.increment(dE33, dt)
        e1.record(st)
        _, nn = solver.nucleate(s)
        _, ps = solver.pf_step(pf_steps)
        e2.record(st)
        e2.synchronize()
        out.append(dict(evp_ms=e0.elapsed_time(e1), step_ms=e0.elapsed_time(e2), it=es.iterations,
                        sig33=es.sig_mean[2], nuclei=nn, X_rex=ps.X_rex, F=ps.F_tot, n_grains=ps.n_grains,
                        rc=rc))
    return out


def native(args, ws, rank, local):
    import torch
    from paper_1509_04953_gb300 import build, evp
    build.build()
    torch.cuda.set_device(local)
    wl = synth.WORKLOADS[args.workload]
    mat = synth.Material()
    seeds, quat = workload_inputs(wl)
    g0 = evp.voronoi(wl.n, seeds).cpu().numpy()
    N3 = wl.n ** 3
    tol_main = args.tol64 if args.precision == "fp64" else args.tol
    mixed = evp.Solver(wl.n, wl.grains, g0, quat, mat, wl.seed, precision=args.precision, tol=tol_main, max_iter=5000,
                       newton_adapt=args.newton_adapt, newton_tol=args.newton_tol, ref_scale=args.ref_scale)
    # warm-up (untimed)
    warm = run_steps(mixed, args.warmup, wl.dE33, wl.dt, wl.pf_steps, torch)
    # inside the timed region only the local solve (the roofline's kernel) is bracketed by CUDA events: events
    # around all seven launches of an iteration cost about 10 % of the step
    mixed.set_profiling_classes(["newton"])
    mixed.kernel_times(reset=True)
    l0 = mixed.launch_count()
    n0 = mixed.newton_counts()
    clocks = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    timed = run_steps(mixed, args.steps, wl.dE33, wl.dt, wl.pf_steps, torch)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    barrier(ws)
    clk = clocks.stop()
    ktimes = mixed.kernel_times(reset=True)
    launches = mixed.launch_count() - l0
    n1 = mixed.newton_counts()
    # the split over all kernel classes: one more increment with every launch bracketed, after the timed region
    mixed.set_profiling(True)
    split_steps = run_steps(mixed, 1, wl.dE33, wl.dt, wl.pf_steps, torch)
    ksplit = mixed.kernel_times(reset=True)
    mixed.set_profiling(False)
    evp_s = sum(r["evp_ms"] for r in timed) / 1e3
    step_s = sum(r["step_ms"] for r in timed) / 1e3
    iters = sum(r["it"] for r in timed)
    step_s_max = allreduce_max(step_s, ws)
    evp_s_max = allreduce_max(evp_s, ws)
    tot_iters = allreduce_sum(iters, ws)
    value = N3 * tot_iters / evp_s_max
    incs_per_s = ws * args.steps / step_s_max

    res = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps, warmup=args.warmup,
               ms_per_step=1e3 * step_s_max / args.steps, higher_is_better=True, scaling="weak",
               vs_baseline=None, dtype={"mixed": "f32 fields/FFT/PF/residual + f64 tangent factorisation and reductions",
                                        "mixed_fast": "f32 (f64 reductions)", "fp64": "f64"}[args.precision],
               data="synthetic",
               config={"workload": wl.name, "n": wl.n, "grains": wl.grains, "precision": args.precision,
                       "tol": tol_main, "newton_tol": mixed.cfg.newton_tol, "newton_adapt": mixed.cfg.newton_adapt,
                       "ref_scale": args.ref_scale,
                       "newton_mode": ["exact", "reuse", "f32_tangent"][mixed.cfg.newton_mode],
                       "dE33": wl.dE33, "pf_steps": wl.pf_steps,
                       "l2": "inputs larger than L2 (about 0.8 GB of fields per replica, no flush needed)",
                       "parallelism": f"replicas x{ws}"},
               drx_increments_per_s=incs_per_s,
               fixed_point_iterations=[r["it"] for r in timed],
               gpu_launches=int(launches), clocks=clk)
    # roofline of the dominant kernel class (timed live over the timed region)
    pk, pk_kind = peaks()
    res["kernel_ms"] = {k: round(v[0], 3) for k, v in ksplit.items() if v[1]}
    res["kernel_launches"] = {k: v[1] for k, v in ksplit.items() if v[1]}
    res["kernel_split_note"] = (f"kernel_ms / kernel_launches: one increment after the timed region "
                                f"({split_steps[0]['it']} iterations) with every launch bracketed by CUDA events")
    dom = max(ksplit, key=lambda k: ksplit[k][0])
    if not ktimes[dom][1]:
        dom = "newton"
    solves, evals = n1[0] - n0[0], n1[1] - n0[1]
    res["newton"] = {"mode": "reuse" if mixed.cfg.newton_mode == 1 else "exact", "solves": solves, "evals": evals, "factorisations": n1[2] - n0[2],
                     "solves_per_voxel_iter": solves / (N3 * iters), "evals_per_voxel_iter": evals / (N3 * iters),
                     "factorisations_per_voxel_iter": (n1[2] - n0[2]) / (N3 * iters)}
    pipes = pipe_peaks(evp)
    res["pipe_peaks_tflops"] = pipes
    res["roofline"] = roofline(dom, ktimes, wl, N3, iters, solves, evals, pk, pk_kind, precision=args.precision,
                               facs=n1[2] - n0[2], reuse=mixed.cfg.newton_mode == 1, pipes=pipes)
    res["memory_bound_kernels"] = memory_kernels(ksplit, wl, N3, args.precision, pk, iterations=split_steps[0]["it"])
    if args.fast_steps > 0:
        res["mixed_fast"] = fast_companion(args, wl, g0, quat, mat, torch, evp)
    if args.soft_ref_steps > 0:
        res["softer_reference_medium"] = soft_ref_companion(args, wl, g0, quat, mat, torch, evp, warm + timed)
    if args.al_steps > 0:
        res["augmented_lagrangian"] = al_companion(args, wl, g0, quat, mat, torch, evp, warm + timed)
    if args.pf2_steps > 0:
        res["pf_grid_2to1"] = pf2_companion(args, wl, g0, quat, mat, torch, evp, pk)
    if args.mr_steps > 0:
        res["ma_roters"] = mr_companion(args, wl, g0, quat, torch, evp, pk)
    if args.fft_reps > 0:
        res["fft_vs_cufft"] = fft_comparator(wl, torch, evp, args.fft_reps, pk)
    if args.trajectory > 0:
        res["trajectory"] = trajectory_companion(args, wl, g0, quat, mat, torch, evp)
    if args.large_steps > 0:
        res["large_256"] = large_companion(args, torch, evp, pk)
    # FP64 companion run on the same seeded input (the full-run comparison above supersedes it by default)
    n64 = (0 if args.trajectory > 0 else args.warmup + args.steps) if args.fp64_steps < 0 else args.fp64_steps
    if n64 > 0:
        res["fp64"] = fp64_companion(args, wl, g0, quat, mat, n64, warm + timed, torch, evp)
    if not args.no_e2e:
        res["e2e"] = e2e(mixed, wl, torch, evp)
    del mixed
    return res


# Measured DRAM traffic (ncu dram__bytes_read.sum + dram__bytes_write.sum, averaged over 20 iterations of the
# second increment, where pass 1 takes one step) of one local-solve iteration (pass 1 326.8 MB + pass 2 0.06 MB;
# the two-step pass 1 of an increment's first iterations moves 327.9 MB), per workload, with the SHA-256 prefix of
# the local-solve sources it was taken on. A figure taken on other sources is stale and reported as null.
NEWTON_TRAFFIC = {(128, "mixed", True): (326.8e6, "e2768457d0fe49dd")}
NEWTON_SOURCES = ("paper_1509_04953_gb300/csrc/newton.cu", "paper_1509_04953_gb300/csrc/local.cuh")


def sources_sha(paths):
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(table, key, paths):
    """The stored ncu traffic for `key` if it was taken on the current sources, else None."""
    entry = table.get(key)
    if entry is None:
        return None
    value, sha = entry
    return value if sha == sources_sha(paths) else None


def hbm_bytes_per_voxel(kernel, n, T):
    """Algorithmic HBM bytes per voxel for one launch of a memory-bound kernel (each field word read
    and written once; half spectra have (n/2+1)/n complex words per real word)."""
    Hw = (n // 2 + 1) / n
    return {"fft_xy_r2c": (6 + 12 * Hw) * T, "fft_y_fwd": 24 * Hw * T, "fft_z_gamma": 24 * Hw * T,
            "fft_y_inv": 24 * Hw * T, "fft_xy_c2r_update": (12 * Hw + 12) * T,
            "predictor": (12 + 6 + 6 + 6 + 1) * T, "state_update": (6 + 1 + 6 + 4 * 6 + 24) * T + 4 + 8,
            "pf_step": 2 * 8 * (4 + T) + 8}.get(kernel)


def pipe_peaks(evp):
    """FP32 and FP64 FMA-pipe throughput of this GPU, measured by the library's own FMA-chain kernel (best of
    three runs each), with the nominal figures as the fallback."""
    out = {}
    for name, nominal in (("fp32", FP32_PEAK_TFLOPS), ("fp64", FP64_PEAK_TFLOPS)):
        try:
            out[name] = max(evp.fma_throughput(name) for _ in range(3))
            out[name + "_source"] = "measured (evp_fma_throughput)"
        except Exception as e:   # noqa: BLE001 -- report the nominal figure and why
            out[name] = nominal
            out[name + "_source"] = f"nominal ({e})"
    return out


def roofline(dom, ktimes, wl, N3, iters, solves, evals, pk, pk_kind, precision, facs=0, reuse=False, pipes=None):
    ms, n = ktimes[dom]
    avg_s = per_unit(dom, ms, n, iters)
    T = 4 if precision != "fp64" else 8
    if dom == "newton":
        # Count the algorithmic flops by pipe and report the pipe they bind. Tangent reuse (chord)
        # does one tangent evaluation and one FP64 factorisation per refresh and residual-only
        # evaluations otherwise; its stored factors are applied in the field precision. The exact
        # Newton evaluates the tangent every time and factorises and solves in FP64 on the mixed
        # path, in FP32 on the fast mixed path.
        if reuse:
            ev = NEWTON_FLOPS_RESID * (evals - facs) + NEWTON_FLOPS_EVAL * facs
            f64 = NEWTON_FLOPS_FACTOR * facs + (NEWTON_FLOPS_SOLVE * solves if precision == "fp64" else 0)
            f32 = (NEWTON_FLOPS_SOLVE * solves if precision != "fp64" else 0)
        else:
            ev = NEWTON_FLOPS_EVAL * evals
            lin = (NEWTON_FLOPS_FACTOR + NEWTON_FLOPS_SOLVE) * solves
            f64, f32 = (lin, 0) if precision in ("mixed", "fp64") else (0, lin)
        if precision == "fp64":
            f64 += ev
        else:
            f32 += ev
        p32 = (pipes or {}).get("fp32", FP32_PEAK_TFLOPS)
        p64 = (pipes or {}).get("fp64", FP64_PEAK_TFLOPS)
        t64, t32 = f64 / p64, f32 / p32
        flops, peak, pipe = (f64, p64, "fp64") if t64 >= t32 else (f32, p32, "fp32")
        alu = flops / (ms / 1e3) / 1e12
        # algorithmic HBM bytes per launch, the method's operands of the local update (Eqs. HookeLaw and
        # PlasticRate): total strain 6, plastic strain 6, the 12 critical resolved shear stresses, the grain id and
        # the stress warm start 6 read, the stress 6 written. Stored tangent factors are this implementation's
        # cache, not the method's work, and are not counted; the formulation's minimal operands (trial strain 6,
        # stress 6, one tau_c, grain id -> stress 6) and the bytes with the factor cache are given as context.
        words = 6 + 6 + 12 + 6 + 6
        bytes_launch = (words * T + 4) * N3
        minimal_launch = ((6 + 6 + 1 + 6) * T + 4) * N3
        with_cache_launch = ((6 + 6 + 1 + (21 if reuse else 0) + 6) * T + 4) * N3
        hbm = bytes_launch / avg_s / 1e9
        hpk = pk.get("hbm_gbs", 6800.0)
        alu_frac, hbm_frac = alu / peak, hbm / hpk
        detail = {"alu": {"pipe": pipe, "achieved": alu, "peak": peak, "unit": "TFLOP/s", "frac": alu_frac,
                          "flops_fp32": f32, "flops_fp64": f64},
                  "hbm": {"achieved": hbm, "peak": hpk, "unit": "GB/s", "frac": hbm_frac,
                          "bytes_per_launch": bytes_launch, "peak_source": pk_kind,
                          "minimal_operand_bytes_per_launch": minimal_launch,
                          "frac_by_minimal_operands": minimal_launch / avg_s / 1e9 / hpk,
                          "bytes_per_launch_with_factor_cache": with_cache_launch}}
        top = detail["hbm"] if hbm_frac >= alu_frac else detail["alu"]
        # DRAM bytes of one local-solve iteration (both passes) from an ncu capture at this workload, when one was
        # taken on the current sources
        traffic = measured_traffic(NEWTON_TRAFFIC, (wl.n, precision, reuse), NEWTON_SOURCES)
        return {"bound": "hbm" if hbm_frac >= alu_frac else "alu", "kernel": "newton",
                "achieved": top["achieved"], "peak": top["peak"], "unit": top["unit"], "frac": top["frac"],
                "traffic": traffic, "traffic_unit": "bytes per launch", "resources": detail,
                "note": "the local solve is reported against the resource it uses the larger fraction of. "
                        "Algorithmic flops: 1140 per residual+tangent evaluation, 544 per residual-only "
                        "evaluation, 80 per 6x6 LDL^T factorisation, 72 per pair of triangular solves, counted "
                        "by pipe, pipe peaks measured in the same run (evp_fma_throughput); algorithmic bytes: the "
                        "method's per-voxel operands (strain, plastic strain, 12 critical stresses, grain id, "
                        "stress warm start -> stress: 148 B FP32), read and written once per launch"}
    if hbm_bytes_per_voxel(dom, wl.n, T) is None:
        return {"bound": "unknown", "kernel": dom, "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None}
    b = hbm_bytes_per_voxel(dom, wl.n, T) * N3
    achieved = b / avg_s / 1e9
    peak = pk.get("hbm_gbs", 6800.0)
    return {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None, "peak_source": pk_kind}


# Kernel classes launched once per fixed-point iteration. Iterations are queued in batches and the ones queued after
# convergence return at once, so these classes are averaged over the iterations that ran, not over their launches.
ITERATION_CLASSES = ("newton", "fft_xy_r2c", "fft_y_fwd", "fft_z_gamma", "fft_y_inv", "fft_xy_c2r_update")


def per_unit(kernel, ms, launches, iterations):
    """Average time of one unit of work of a kernel class, in seconds: one iteration for the iteration classes (the
    time of the brackets that returned at once counts against the iterations that ran), one launch otherwise."""
    units = iterations if (kernel in ITERATION_CLASSES and iterations) else launches
    return ms / 1e3 / max(units, 1)


def memory_kernels(ktimes, wl, N3, precision, pk, iterations=None):
    T = 4 if precision != "fp64" else 8
    out = {}
    for k, (ms, n) in ktimes.items():
        bpv = hbm_bytes_per_voxel(k, wl.n, T)
        if bpv is None or n == 0:
            continue
        avg = per_unit(k, ms, n, iterations)
        gbs = bpv * N3 / avg / 1e9
        out[k] = {"avg_us": round(1e6 * avg, 2), "GB/s": round(gbs, 1), "frac": round(gbs / pk.get("hbm_gbs", 6800.0), 3)}
    return out


def fft_comparator(wl, torch, evp, reps, pk):
    """The library's 3D real-to-complex and complex-to-real FFTs of six FP32 fields (the stress / strain
    spectra of one fixed-point iteration, without the fused Green operator) against cuFFT through torch.fft,
    same data, same stream, CUDA events over `reps` repetitions after a warm-up."""
    n = wl.n
    g = torch.Generator(device="cuda").manual_seed(wl.seed)
    x = torch.randn((6, n, n, n), device="cuda", dtype=torch.float32, generator=g)
    st = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        b.synchronize()
        return 1e3 * a.elapsed_time(b) / reps

    spec = evp.rfft3d(x)
    ours_f = timed(lambda: evp.rfft3d(x))
    ours_i = timed(lambda: evp.irfft3d(spec.clone()))
    clone_us = timed(lambda: spec.clone())
    cu_f = timed(lambda: torch.fft.rfftn(x, dim=(1, 2, 3)))
    sc = torch.fft.rfftn(x, dim=(1, 2, 3))
    # unnormalised inverse on both sides (norm="forward" leaves the inverse unscaled)
    cu_i = timed(lambda: torch.fft.irfftn(sc, s=(n, n, n), dim=(1, 2, 3), norm="forward"))
    err = (spec - sc).abs().max().item() / sc.abs().max().item()
    ours_i -= clone_us   # the inverse consumes its input: a copy per repetition, subtracted
    H = n // 2 + 1
    b = 6 * (n ** 3 * 4 + n * n * H * 8) * 3   # three passes, each reading and writing the fields once
    out = {"fields": 6, "n": n, "reps": reps,
           "ours_forward_us": round(ours_f, 1), "ours_inverse_us": round(ours_i, 1),
           "cufft_forward_us": round(cu_f, 1), "cufft_inverse_us": round(cu_i, 1),
           "speedup_vs_cufft": round((cu_f + cu_i) / (ours_f + ours_i), 3),
           "spectrum_rel_diff_vs_cufft": err,
           "ours_forward_GB/s_3_passes": round(b / (ours_f * 1e-6) / 1e9, 1),
           "note": "forward and inverse of six 128^3 FP32 fields; inside the fixed point the Green operator, the "
                   "residual and the control ride in the z pass and the strain update in the x pass"}
    return out


def soft_ref_companion(args, wl, g0, quat, mat, torch, evp, main_hist):
    """The same increments with the basic scheme's reference shear modulus mu_Voigt / soft_ref (Voigt bulk): the
    same converged solution (macro stress compared with the main run's, increment by increment) in fewer
    iterations; timed over the last soft_ref_steps increments."""
    s = evp.Solver(wl.n, wl.grains, g0, quat, mat, wl.seed, precision=args.precision,
                   tol=args.tol64 if args.precision == "fp64" else args.tol, max_iter=5000,
                   newton_adapt=args.newton_adapt, newton_tol=args.newton_tol, ref_scale=args.soft_ref)
    w = max(len(main_hist) - args.soft_ref_steps, 0)
    hw = run_steps(s, w, wl.dE33, wl.dt, wl.pf_steps, torch)
    h = run_steps(s, args.soft_ref_steps, wl.dE33, wl.dt, wl.pf_steps, torch)
    evp_s = sum(r["evp_ms"] for r in h) / 1e3
    step_s = sum(r["step_ms"] for r in h) / 1e3
    errs = [abs(a["sig33"] - b["sig33"]) / abs(b["sig33"]) for a, b in zip(hw + h, main_hist)]
    return {"ref_scale": args.soft_ref, "voxel_iters_per_s": wl.n ** 3 * sum(r["it"] for r in h) / evp_s,
            "drx_increments_per_s": len(h) / step_s, "ms_per_step": 1e3 * step_s / len(h),
            "fixed_point_iterations": [r["it"] for r in hw + h],
            "main_run_iterations": [r["it"] for r in main_hist],
            "macro_stress_rel_diff_vs_main_max": max(errs)}


def fast_companion(args, wl, g0, quat, mat, torch, evp):
    """The mixed path with the 6x6 Newton solve in FP32 (EVP_MIXED_FAST), same input."""
    s = evp.Solver(wl.n, wl.grains, g0, quat, mat, wl.seed, precision="mixed_fast", tol=args.tol, max_iter=5000,
                   newton_adapt=args.newton_adapt, ref_scale=args.ref_scale)
    run_steps(s, 1, wl.dE33, wl.dt, wl.pf_steps, torch)
    h = run_steps(s, args.fast_steps, wl.dE33, wl.dt, wl.pf_steps, torch)
    evp_s = sum(r["evp_ms"] for r in h) / 1e3
    step_s = sum(r["step_ms"] for r in h) / 1e3
    return {"voxel_iters_per_s": wl.n ** 3 * sum(r["it"] for r in h) / evp_s,
            "drx_increments_per_s": len(h) / step_s, "increments": len(h),
            "fixed_point_iterations": [r["it"] for r in h]}


def pf2_companion(args, wl, g0, quat, mat, torch, evp, pk):
    """The same increments with the phase field on the paper's 2:1 grid ((2n)^3 PF points): DRX
    increments/s and the live cost of one PF step there, against its algorithmic bytes."""
    s = evp.Solver(wl.n, wl.grains, g0, quat, mat, wl.seed, precision=args.precision,
                   tol=args.tol64 if args.precision == "fp64" else args.tol, max_iter=5000,
                   newton_adapt=args.newton_adapt, pf_refine=2, ref_scale=args.ref_scale)
    run_steps(s, 1, wl.dE33, wl.dt, wl.pf_steps, torch)
    s.set_profiling_classes(["pf_step"])
    s.kernel_times(reset=True)
    h = run_steps(s, args.pf2_steps, wl.dE33, wl.dt, wl.pf_steps, torch)
    kt = s.kernel_times(reset=True)
    step_s = sum(r["step_ms"] for r in h) / 1e3
    T = 4 if args.precision != "fp64" else 8
    M3 = (2 * wl.n) ** 3
    ms, nl = kt.get("pf_step", (0.0, 0))
    out = {"pf_points": M3, "drx_increments_per_s": len(h) / step_s, "ms_per_step": 1e3 * step_s / len(h),
           "increments": len(h), "X_rex": h[-1]["X_rex"], "n_grains": h[-1]["n_grains"]}
    if nl:
        # PF launches include one interpolation of the driving force per call
        steps = nl - len(h)
        per = ms / max(steps, 1) / 1e3
        b = hbm_bytes_per_voxel("pf_step", wl.n, T) * M3
        out["pf_step_us"] = round(1e6 * per, 1)
        out["pf_step_GB/s"] = round(b / per / 1e9, 1)
        out["pf_step_frac"] = round(b / per / 1e9 / pk.get("hbm_gbs", 6800.0), 3)
    return out


MR_DT_PER_STRAIN = 625.0   # s per unit strain: the paper's strain rate 1.6e-3 /s


def mr_bytes_per_voxel(T):
    """Algorithmic HBM bytes per voxel of the Ma-Roters state update (three launches): shear rates and
    strains (reads sigma 6, tau_pass and 1/tau_cut 24, trial / elastic / plastic strain 18, grain id; writes
    eps_p, eps_e, strain increment 18, rates 12, (sigma_vm, gdot_vm) 2), the density update (reads the rates
    12, aux 2, sigma 6, SSD / GND 48, both grain ids; writes SSD / GND 48) and k (reads 48, writes k)."""
    return (6 + 24 + 18 + 18 + 12 + 2) * T + 4 + (12 + 2 + 6 + 48 + 48) * T + 8 + 48 * T + 8


def mr_companion(args, wl, g0, quat, torch, evp, pk):
    """The paper's own constitutive law (Ma-Roters, Sec. 2.2) on the same grid and grains, with the
    augmented-Lagrangian solver the paper names, at the paper's strain rate (1e-3 strain per increment in
    0.625 s): throughput, the live rate of the local solve and of the density update against their
    algorithmic bytes, and the mixed path's macro stress against the FP64 path's."""
    mat = synth.ma_roters_material()
    dt = abs(wl.dE33) * MR_DT_PER_STRAIN
    prec = args.precision
    tol = args.tol64 if prec == "fp64" else 5e-6
    s = evp.Solver(wl.n, wl.grains, g0, quat, mat, wl.seed, precision=prec, law="mr", scheme="al", al_scale=8.0,
                   tol=tol, max_iter=5000)
    hw = run_steps(s, 1, wl.dE33, dt, wl.pf_steps, torch)
    s.set_profiling_classes(["newton", "state_update"])   # the two classes reported below
    s.kernel_times(reset=True)
    n0 = s.newton_counts()
    h = run_steps(s, args.mr_steps, wl.dE33, dt, wl.pf_steps, torch)
    kt = s.kernel_times(reset=True)
    n1 = s.newton_counts()
    N3 = wl.n ** 3
    T = 4 if prec != "fp64" else 8
    evp_s = sum(r["evp_ms"] for r in h) / 1e3
    step_s = sum(r["step_ms"] for r in h) / 1e3
    iters = sum(r["it"] for r in h)
    hpk = pk.get("hbm_gbs", 6800.0)
    out = {"law": "Ma-Roters (Eqs. FlowRule, RhoForest, RhoParallel, SSDEvolution, GNDEvolution, L0evolution)",
           "scheme": "augmented Lagrangian, al_scale 8", "precision": prec, "tol": tol, "dt": dt,
           "voxel_iters_per_s": N3 * iters / evp_s, "drx_increments_per_s": len(h) / step_s,
           "ms_per_step": 1e3 * step_s / len(h), "increments": len(h),
           "fixed_point_iterations": [r["it"] for r in hw + h], "sig33": [round(r["sig33"], 4) for r in hw + h],
           "leff_m": s.leff, "kernel_ms": {k: round(v[0], 3) for k, v in kt.items() if v[1]},
           "newton_solves_per_voxel_iter": (n1[0] - n0[0]) / (N3 * max(iters, 1)),
           "newton_evals_per_voxel_iter": (n1[1] - n0[1]) / (N3 * max(iters, 1))}
    ms, nl = kt.get("state_update", (0.0, 0))
    if nl:
        per = ms / len(h) / 1e3
        b = mr_bytes_per_voxel(T) * N3
        out["state_update"] = {"us_per_increment": round(1e6 * per, 1), "GB/s": round(b / per / 1e9, 1),
                               "frac": round(b / per / 1e9 / hpk, 3), "bytes_per_increment": b}
    ms, nl = kt.get("newton", (0.0, 0))
    if nl:
        per = per_unit("newton", ms, nl, iters)
        # AL local step, per voxel: reads trial and elastic strain, multiplier, stress (24), tau_ref (1), tau_pass
        # and 1/tau_cut (24), stored factors (24 planes' words) and the grain id; writes stress, multiplier,
        # polarisation (18) and, on a refresh, the factors
        b = ((6 + 6 + 6 + 6 + 1 + 24 + 24 + 18) * T + 4) * N3
        out["local_solve"] = {"us_per_iteration": round(1e6 * per, 1), "GB/s": round(b / per / 1e9, 1),
                              "frac": round(b / per / 1e9 / hpk, 3)}
    if args.mr_fp64_steps > 0 and prec != "fp64":
        s64 = evp.Solver(wl.n, wl.grains, g0, quat, mat, wl.seed, precision="fp64", law="mr", scheme="al",
                         al_scale=8.0, tol=args.tol64, max_iter=5000)
        h64 = run_steps(s64, min(args.mr_fp64_steps, len(hw + h)), wl.dE33, dt, wl.pf_steps, torch)
        errs = [abs(a["sig33"] - b["sig33"]) / abs(b["sig33"]) for a, b in zip(hw + h, h64)]
        e64 = sum(r["evp_ms"] for r in h64) / 1e3
        out["fp64"] = {"voxel_iters_per_s": N3 * sum(r["it"] for r in h64) / e64,
                       "fixed_point_iterations": [r["it"] for r in h64], "tol": args.tol64,
                       "mixed_vs_fp64_macro_stress_rel_err_max": max(errs)}
        del s64
    del s
    return out


def mr_oracle_sample(wl, dt, iters_cap):
    """The FP64 oracle on the same Ma-Roters increment (augmented Lagrangian), capped at `iters_cap` iterations:
    the CPU rate beside the GPU's, in the same unit."""
    import oracle as O
    seeds, quat = workload_inputs(wl)
    g0 = O.voronoi(wl.n, seeds)
    st = O.State(wl.n, wl.grains, g0, quat, synth.ma_roters_material(), seed=wl.seed, tol=0.0, max_iter=iters_cap,
                 allow_unconverged=1, scheme=1, al_scale=8.0, law=1, nthreads=cpu_cores())
    t0 = time.perf_counter()
    rc, s = st.increment(wl.dE33, dt)
    t1 = time.perf_counter()
    st.close()
    return {"voxel_iters_per_s": wl.n ** 3 * s.iterations / (t1 - t0), "cores": cpu_cores(), "kind": "oracle",
            "sample": f"one {wl.n}^3 Ma-Roters increment capped at {s.iterations} augmented-Lagrangian iterations "
                      f"(FP64, OpenMP over voxels; includes the initial local solve), {t1 - t0:.1f} s"}


def al_companion(args, wl, g0, quat, mat, torch, evp, basic_hist):
    """The augmented-Lagrangian solver (the scheme the paper names) on the same input and precision:
    increments 1..W+K, timed over the last K, macro stress compared with the basic scheme."""
    s = evp.Solver(wl.n, wl.grains, g0, quat, mat, wl.seed, precision=args.precision,
                   tol=args.tol64 if args.precision == "fp64" else args.tol, max_iter=5000, scheme="al")
    w = len(basic_hist) - args.steps
    hw = run_steps(s, w, wl.dE33, wl.dt, wl.pf_steps, torch)
    s.set_profiling_classes(["newton"])
    s.kernel_times(reset=True)
    h = run_steps(s, args.steps, wl.dE33, wl.dt, wl.pf_steps, torch)
    kt = s.kernel_times(reset=True)
    evp_s = sum(r["evp_ms"] for r in h) / 1e3
    step_s = sum(r["step_ms"] for r in h) / 1e3
    errs = [abs(a["sig33"] - b["sig33"]) / abs(b["sig33"]) for a, b in zip(hw + h, basic_hist)]
    return {"voxel_iters_per_s": wl.n ** 3 * sum(r["it"] for r in h) / evp_s,
            "drx_increments_per_s": len(h) / step_s, "ms_per_step": 1e3 * step_s / len(h),
            "fixed_point_iterations": [r["it"] for r in hw + h], "al_scale": 6.0,
            "macro_stress_rel_diff_vs_basic_max": max(errs),
            "kernel_ms": {k: round(v[0], 3) for k, v in kt.items() if v[1]}}


def fp64_companion(args, wl, g0, quat, mat, nsteps, mixed_hist, torch, evp):
    s64 = evp.Solver(wl.n, wl.grains, g0, quat, mat, wl.seed, precision="fp64", tol=args.tol64, max_iter=5000,
                     ref_scale=args.ref_scale)
    h = run_steps(s64, nsteps, wl.dE33, wl.dt, wl.pf_steps, torch)
    N3 = wl.n ** 3
    m = mixed_hist[:nsteps]
    errs = [abs(a["sig33"] - b["sig33"]) / abs(b["sig33"]) for a, b in zip(m, h)]
    evp_s = sum(r["evp_ms"] for r in h) / 1e3
    step_s = sum(r["step_ms"] for r in h) / 1e3
    out = {"voxel_iters_per_s": N3 * sum(r["it"] for r in h) / evp_s, "drx_increments_per_s": nsteps / step_s,
           "ms_per_step": 1e3 * step_s / nsteps, "increments": nsteps,
           "fixed_point_iterations": [r["it"] for r in h], "tol": args.tol64,
           "mixed_vs_fp64_macro_stress_rel_err_max": max(errs),
           "X_rex_abs_diff_max": max(abs(a["X_rex"] - b["X_rex"]) for a, b in zip(m, h))}
    return out


def one_increment(solver, step, dE33, dt, pf_steps, torch):
    """One DRX increment (solve, nucleation, PF steps) bracketed by CUDA events on the solver's stream."""
    st = solver.stream
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(st)
    rc, es = solver.increment(dE33, dt)
    e1.record(st)
    _, nn = solver.nucleate(step)
    _, ps = solver.pf_step(pf_steps)
    e2.record(st)
    e2.synchronize()
    return dict(evp_ms=e0.elapsed_time(e1), step_ms=e0.elapsed_time(e2), it=es.iterations, sig33=es.sig_mean[2],
                nuclei=nn, X_rex=ps.X_rex, F=ps.F_tot, n_grains=ps.n_grains, overflow=ps.overflow, rc=rc)


def field_errors(mixed, fp64):
    """The mixed path's voxel stress field against the FP64 path's: max and RMS difference, relative to the
    largest mean-stress component and to the FP64 field's RMS, over all voxels and over the voxels whose grain id
    agrees (DRX events can differ near a nucleation threshold: k differs between precisions in its last bits)."""
    sm = mixed.get("sig").astype(np.float64)
    sd = fp64.get("sig")
    d = sm - sd
    den = float(np.abs(sd.mean(axis=1)).max())
    same = mixed.get("g")[0] == fp64.get("g")[0]
    dsame = d[:, same]
    return {"max_rel_to_mean": float(np.abs(d).max() / den), "rms_rel_to_mean": float(np.sqrt((d ** 2).mean()) / den),
            "rms_rel": float(np.sqrt((d ** 2).sum() / (sd ** 2).sum())),
            "rms_rel_same_grain": float(np.sqrt((dsame ** 2).sum() / (sd[:, same] ** 2).sum())),
            "max_rel_to_mean_same_grain": float(np.abs(dsame).max() / den),
            "same_grain_fraction": float(same.mean())}


def trajectory_companion(args, wl, g0, quat, mat, torch, evp):
    """The whole workload (wl.increments increments, to strain |dE33| x increments), FP32-mixed and FP64 on the same
    seeded input in lockstep: the mixed path's error against FP64 on the macroscopic stress-strain curve, the voxel
    stress field (every `every` increments) and the recrystallised fraction; the mixed path's throughput over the
    whole run and over a window taken in the DRX regime; the DRX analytics (critical strain, Avrami fit, grains as
    connected components) of both runs."""
    from paper_1509_04953_gb300 import analytics as A
    T = args.trajectory
    N3 = wl.n ** 3
    # every boundary voxel can nucleate again in every increment once k exceeds the redrawn strengths (reading
    # C17): the grain-id space is sized for the whole run
    ids = min(wl.grains + 64 * N3, 2 ** 31 - 1)
    kw = dict(precision=args.precision, tol=args.tol, max_iter=5000, newton_adapt=args.newton_adapt,
              newton_tol=args.newton_tol, ref_scale=args.ref_scale, max_ids=ids)
    mx = evp.Solver(wl.n, wl.grains, g0, quat, mat, wl.seed, **kw)
    f64 = evp.Solver(wl.n, wl.grains, g0, quat, mat, wl.seed, precision="fp64", tol=args.tol64, max_iter=20000,
                     scheme=args.trajectory_fp64_scheme, max_ids=ids)
    # the mixed path restarted from the FP64 state at each checkpoint: the error of one increment from a common
    # state, free of the divergence of the two runs' discrete DRX histories
    scratch = evp.Solver(wl.n, wl.grains, g0, quat, mat, wl.seed, **kw)
    state_fields = ("sig", "epse", "epsp", "deps", "rho")
    hm, hd, fields, common = [], [], [], []
    every = max(T // 10, 1)
    synced = False
    for t in range(T):
        hm.append(one_increment(mx, t, wl.dE33, wl.dt, wl.pf_steps, torch))
        if synced:
            _, sc = scratch.increment(wl.dE33, wl.dt)
        hd.append(one_increment(f64, t, wl.dE33, wl.dt, wl.pf_steps, torch))
        if synced:
            sd = f64.get("sig")
            d = scratch.get("sig").astype(np.float64) - sd
            common.append({"increment": t + 1, "macro_rel": abs(sc.sig_mean[2] - hd[-1]["sig33"]) / abs(hd[-1]["sig33"]),
                           "voxel_sigma_rms_rel": float(np.sqrt((d ** 2).sum() / (sd ** 2).sum())),
                           "voxel_sigma_max_rel_to_mean": float(np.abs(d).max() / np.abs(sd.mean(axis=1)).max())})
            synced = False
        if (t + 1) % every == 0 or t + 1 == T:
            fe = field_errors(mx, f64)
            fe["increment"] = t + 1
            fe["strain"] = (t + 1) * abs(wl.dE33)
            fe["curve_rel"] = abs(hm[-1]["sig33"] - hd[-1]["sig33"]) / abs(hd[-1]["sig33"])
            fields.append(fe)
            if t + 1 < T:
                for f in state_fields:
                    scratch.set(f, f64.get(f))
                sc64 = f64.scalars()
                scratch.set_scalars(sc64["E"], sc64["dE_prev"], sc64["have_prev"], sc64["next_id"])
                synced = True
    strain = [(t + 1) * abs(wl.dE33) for t in range(T)]
    curve_err = [abs(a["sig33"] - b["sig33"]) / abs(b["sig33"]) for a, b in zip(hm, hd)]
    xr_err = [abs(a["X_rex"] - b["X_rex"]) for a, b in zip(hm, hd)]
    # DRX window: the mixed path's increments from the first one at or past X_rex = 0.1, or the last quarter
    w0 = next((i for i, r in enumerate(hm) if r["X_rex"] >= 0.1), 3 * T // 4)
    w0 = min(w0, max(T - args.drx_window, 0))
    win = hm[w0:w0 + args.drx_window]
    wstep = sum(r["step_ms"] for r in win) / 1e3
    wevp = sum(r["evp_ms"] for r in win) / 1e3

    def analytics(h, solver):
        out = {"critical_strain": A.critical_strain(strain, [r["nuclei"] for r in h])}
        tt = np.array(strain) / abs(wl.dE33) * wl.dt
        X = np.array([r["X_rex"] for r in h])
        try:
            m, K = A.avrami_fit(tt, X)
            out["avrami"] = {"m": m, "K": K}
        except ValueError as e:
            out["avrami"] = str(e)
        ng, d = A.grain_statistics(solver.get("g")[0], wl.n, dx=mat.dx)
        out["grains_connected"] = ng
        out["mean_diameter_um"] = d * 1e6
        out["n_grains_ids"] = h[-1]["n_grains"]
        return out

    out = {"increments": T, "strain_final": strain[-1], "fp64_scheme": args.trajectory_fp64_scheme,
           "fp64_tol": args.tol64, "mixed_tol": args.tol,
           "mixed_vs_fp64": {"curve_rel_err_max": max(curve_err), "curve_rel_err_final": curve_err[-1],
                             "voxel_sigma": fields, "voxel_sigma_rms_rel_max": max(f["rms_rel"] for f in fields),
                             "voxel_sigma_rms_rel_same_grain_max": max(f["rms_rel_same_grain"] for f in fields),
                             "X_rex_abs_diff_max": max(xr_err), "X_rex_final": [hm[-1]["X_rex"], hd[-1]["X_rex"]],
                             "one_increment_from_common_state": common,
                             "one_increment_voxel_sigma_rms_rel_max": max((c["voxel_sigma_rms_rel"] for c in common),
                                                                          default=None),
                             "one_increment_macro_rel_max": max((c["macro_rel"] for c in common), default=None)},
           "mixed_full_run": {"voxel_iters_per_s": N3 * sum(r["it"] for r in hm) / (sum(r["evp_ms"] for r in hm) / 1e3),
                              "drx_increments_per_s": T / (sum(r["step_ms"] for r in hm) / 1e3),
                              "fixed_point_iterations_total": sum(r["it"] for r in hm),
                              "nuclei_total": sum(r["nuclei"] for r in hm)},
           "drx_window": {"first_increment": w0 + 1, "increments": len(win), "strain": strain[w0],
                          "X_rex": [win[0]["X_rex"], win[-1]["X_rex"]], "nuclei": sum(r["nuclei"] for r in win),
                          "n_grains": win[-1]["n_grains"], "drx_increments_per_s": len(win) / wstep,
                          "voxel_iters_per_s": N3 * sum(r["it"] for r in win) / wevp,
                          "ms_per_step": 1e3 * wstep / len(win),
                          "pf_ms_per_increment": 1e3 * (wstep - wevp) / len(win)},
           "fp64_full_run": {"voxel_iters_per_s": N3 * sum(r["it"] for r in hd) / (sum(r["evp_ms"] for r in hd) / 1e3),
                             "drx_increments_per_s": T / (sum(r["step_ms"] for r in hd) / 1e3)},
           "analytics": {"mixed": analytics(hm, mx), "fp64": analytics(hd, f64)},
           "curve": {"every": every, "strain": strain[every - 1::every],
                     "sig33_mixed": [round(r["sig33"], 4) for r in hm[every - 1::every]],
                     "X_rex_mixed": [r["X_rex"] for r in hm[every - 1::every]],
                     "X_rex_fp64": [r["X_rex"] for r in hd[every - 1::every]],
                     "iterations_mixed": [r["it"] for r in hm[every - 1::every]]}}
    del mx, f64, scratch
    return out


def large_companion(args, torch, evp, pk):
    """The large workload (256^3, 1024 grains, FP32-mixed, 6e-4 strain per 0.6 s increment): DRX increments timed
    after a warm-up, then a checkpointed adjoint sweep over the next `large_adjoint` increments (gradient of the
    summed axial stress with respect to k1, k2, tau0, n), with the forward and adjoint workspace bytes and the
    adjoint workspace that 100 increments with a checkpoint every 10 would take."""
    import ctypes as C
    wl = synth.WORKLOADS["cu256"]
    mat = synth.Material()
    seeds, quat = workload_inputs(wl)
    g0 = evp.voronoi(wl.n, seeds).cpu().numpy()
    s = evp.Solver(wl.n, wl.grains, g0, quat, mat, wl.seed, precision="mixed", tol=args.tol, max_iter=5000)
    ws = evp.workspace_bytes(s.cfg)
    warm = run_steps(s, 2, wl.dE33, wl.dt, wl.pf_steps, torch)
    h = run_steps(s, args.large_steps, wl.dE33, wl.dt, wl.pf_steps, torch)
    N3 = wl.n ** 3
    evp_s = sum(r["evp_ms"] for r in h) / 1e3
    step_s = sum(r["step_ms"] for r in h) / 1e3
    out = {"workload": wl.name, "workspace_bytes": ws, "increments_timed": len(h),
           "voxel_iters_per_s": N3 * sum(r["it"] for r in h) / evp_s, "drx_increments_per_s": len(h) / step_s,
           "ms_per_step": 1e3 * step_s / len(h), "fixed_point_iterations": [r["it"] for r in warm + h],
           "sig33": [round(r["sig33"], 4) for r in warm + h]}
    T = args.large_adjoint
    if T > 0:
        ck = max(1, int(round(T ** 0.5)))
        nb = C.c_size_t(0)
        if evp.load().evp_adjoint_workspace_bytes(C.byref(s.cfg), 100, 10, C.byref(nb)) != 0:
            raise evp.EVPError("evp_adjoint_workspace_bytes refused the 100-increment sweep")
        st = s.stream
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        s.adjoint_begin(T, ck)
        e0.record(st)
        curve = [s.adjoint_step(wl.dE33, wl.dt).sig_mean[2] for _ in range(T)]
        e1.record(st)
        gb = np.zeros((T, 6))
        gb[:, 2] = 1.0                  # L = sum of the axial stresses of the recorded increments
        grad = s.adjoint_end(gb, tol=1e-5)
        e2.record(st)
        e2.synchronize()
        out["adjoint"] = {"increments": T, "checkpoint_every": ck, "workspace_bytes": int(s.adj_ws.numel()),
                          "forward_s": e0.elapsed_time(e1) / 1e3, "reverse_s": e1.elapsed_time(e2) / 1e3,
                          "dL_dtheta": {"k1": grad[0], "k2": grad[1], "tau0": grad[2], "n": grad[3]},
                          "sig33_recorded": [round(c, 4) for c in curve],
                          "workspace_bytes_100_increments_every_10": nb.value}
    s.close()
    return out


def e2e(solver, wl, torch, evp):
    """Same metric through the public C ABI with the state in pinned host memory: every step
    uploads the state fields, runs the increment, nucleation and PF, and downloads them again."""
    names = ["sig", "epse", "epsp", "deps", "rho", "kappa", "g", "draws", "ids", "eta"]
    host = {k: torch.from_numpy(solver.get(k)).pin_memory() for k in names}
    L = evp.load()
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    steps = 5   # the host copies' rate varies from box to box; five steps average it
    st = solver.stream
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    iters = 0
    e0.record(st)
    for s in range(steps):
        for k in names:
            t = host[k]
            rc = L.set_fields(solver.h, evp.FIELDS[k], t.data_ptr(), t.numel() * t.element_size(), 0)
            if rc != 0:
                raise evp.EVPError(f"set_fields({k}): {evp.EVP_ERR.get(rc, rc)}: {solver.last_error()}")
        _, es = solver.increment(wl.dE33, wl.dt)
        iters += es.iterations
        solver.nucleate(100 + s)
        solver.pf_step(wl.pf_steps)
        for k in names:
            t = host[k]
            rc = L.get_fields(solver.h, evp.FIELDS[k], t.data_ptr(), t.numel() * t.element_size(), 0)
            if rc != 0:
                raise evp.EVPError(f"get_fields({k}): {evp.EVP_ERR.get(rc, rc)}: {solver.last_error()}")
    e1.record(st)
    e1.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    return {"value": wl.n ** 3 * iters / secs, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
            "steps": steps, "drx_increments_per_s": steps / secs,
            "note": "state round-trips through pinned host memory every step via set_fields/get_fields"}


# ---------------------------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------------------------
def oracle_sample(wl, iters_cap, nthreads=0):
    """Time the FP64 oracle on the workload: one increment capped at `iters_cap` fixed-point
    iterations (a bounded sample), then nucleation and the phase-field steps."""
    import oracle as O
    mat = synth.Material()
    seeds, quat = workload_inputs(wl)
    g0 = O.voronoi(wl.n, seeds)
    st = O.State(wl.n, wl.grains, g0, quat, mat, seed=wl.seed, tol=0.0, max_iter=iters_cap, allow_unconverged=1,
                 nthreads=nthreads)
    t0 = time.perf_counter()
    rc, s = st.increment(wl.dE33, wl.dt)
    t1 = time.perf_counter()
    st.nucleate(0)
    st.pf_step(wl.pf_steps)
    t2 = time.perf_counter()
    st.close()
    return dict(evp_s=t1 - t0, step_s=t2 - t0, iters=s.iterations)


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def cpu_baseline(wl, mr=False):
    """The oracle timed on the host's cores (bounded samples of the workload, in the metric's unit); with `mr`, also
    on the Ma-Roters increment that the GPU companion runs."""
    cores = cpu_cores()
    r = oracle_sample(wl, 2, nthreads=cores)   # every call sets its own OpenMP thread count
    out = {"value": wl.n ** 3 * r["iters"] / r["evp_s"], "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"one {wl.n}^3 increment capped at {r['iters']} fixed-point iterations (FP64, OpenMP over"
                     f" voxels), {r['evp_s']:.1f} s"}
    # the same on one thread, on the 64^3 / 64-grain configuration (a smaller bounded sample, same unit)
    w64 = synth.WORKLOADS["cu64"]
    r1 = oracle_sample(w64, 1, nthreads=1)
    out["single_thread"] = {"value": w64.n ** 3 * r1["iters"] / r1["evp_s"], "unit": UNIT, "cores": 1,
                            "sample": f"one {w64.n}^3 increment capped at {r1['iters']} fixed-point iteration, "
                                      f"{r1['evp_s']:.1f} s"}
    if mr:
        out["ma_roters"] = mr_oracle_sample(wl, abs(wl.dE33) * MR_DT_PER_STRAIN, 2)
    return out


def reference(args, ws, rank):
    if rank != 0:
        return None
    import oracle
    oracle.build()
    wl = synth.WORKLOADS[args.workload]
    cores = cpu_cores()
    for _ in range(args.warmup):
        oracle_sample(wl, 1)
    evp_s = step_s = 0.0
    iters = 0
    for _ in range(args.steps):
        r = oracle_sample(wl, 1)
        evp_s += r["evp_s"]
        step_s += r["step_s"]
        iters += r["iters"]
    value = wl.n ** 3 * iters / evp_s
    return dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * step_s / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config={"workload": wl.name, "n": wl.n, "grains": wl.grains, "precision": "fp64 (CPU oracle)"},
                cpu_baseline={"value": value, "unit": UNIT, "kind": "oracle", "cores": cores,
                              "sample": f"each step: one {wl.n}^3 increment capped at 1 fixed-point iteration,"
                                        f" nucleation and {wl.pf_steps} phase-field steps"},
                e2e={"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                drx_increments_per_s=None)


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.impl == "reference":
        res = reference(args, ws, rank)
    else:
        res = native(args, ws, rank, local)
        if rank == 0 and ws == 1 and not args.no_cpu_baseline:   # the oracle runs at N = 1 only
            res["cpu_baseline"] = cpu_baseline(synth.WORKLOADS[args.workload], mr=args.mr_steps > 0)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
