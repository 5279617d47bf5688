#!/usr/bin/env python3
"""Benchmark of the Q^k spectral-element fast-diagonalisation solve on GB300.

Workload (one "step" = one full solve of the hot path): Q^4 SEM, 250 elements
per axis on [0,1]^3, n = 999 interior nodes per axis (997,002,999 DoF),
-Lap u + u = f with f from the manufactured u = e^x sin(pi x) sin(pi y)
sin(pi z), homogeneous Dirichlet data.  The headline path is the tcgen05
split-bf16 (BF16x3) solve with 3 FP64 refinement sweeps (error ~1e-13 against
FP64); the plain FP64 DMMA path (+1 FP64 sweep) is timed beside it.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", str(os.cpu_count() or 1))
os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1000^3 Q^4 solve ms & GDoF/s on 1 GB300: FP64 vs refined split-BF16 at 1e-12 err"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def tc_traffic_per_launch(n: int):
    """DRAM bytes (read + write) of one tensor-core pass from the committed ncu
    capture, scaled to n by the DoF processed; None once the kernel source has
    changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_inputs.json")) as fh:
            rec = json.load(fh)
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as fh:
                h.update(fh.read())
        sha = h.hexdigest()
    except (OSError, ValueError, KeyError):
        return None
    if not sha.startswith(rec["source_sha256_prefix"]):
        return None
    px = (n + 15) // 16 * 16
    return rec["dram_bytes_per_launch_n511"] * (px * n * n) / rec["dofs_per_launch_n511"]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return PEAKS_FALLBACK, "fallback"


# --------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[5 + q].lower() == "active"})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


# --------------------------------------------------------------------- oracle baseline

def oracle_sample(n: int, k: int, c: float, lines: int = 63):
    """Time the FP64 oracle (test infrastructure, numpy + BLAS on the host
    cores) on a bounded sample of the n^3 workload: the operations of its
    refined solve (two fast solves of six mode products and one division
    each, one H-form apply), each run on `lines`-thick slabs of full-length
    grid lines.  Every grid line costs the same, so the sample is `lines / n`
    of the refined solve of the whole grid.  Returns (wall seconds of the
    sample, DoF-equivalents it processed = lines * n^2)."""
    from oracle import sem_1d
    from oracle.sem import apply_h, mode_product
    s = sem_1d(k, (n + 1) // k, 0.0, 1.0)
    s_lines = sem_1d(k, (lines + 1) // k, 0.0, 1.0)  # same k: same band cost per node
    rng = np.random.Generator(np.random.PCG64(7))
    slab_xy = rng.standard_normal((lines, n, n))          # (z, y, x): `lines` z-pages
    slab_z = rng.standard_normal((n, lines, n))           # `lines` y-rows, full z
    lam3 = s.lam[:, None, None] + s.lam[None, :, None] + s.lam[None, None, :lines] + c
    t0 = time.perf_counter()
    for _ in range(2):                                    # bare solve, then the refinement solve
        mode_product(slab_z.T, s.Tinv, 2)
        mode_product(slab_xy.T, s.Tinv, 1)
        mode_product(slab_xy.T, s.Tinv, 0)
        _ = slab_xy.T / lam3
        mode_product(slab_xy.T, s.T, 0)
        mode_product(slab_xy.T, s.T, 1)
        mode_product(slab_z.T, s.T, 2)
    apply_h(slab_xy, s, s, s_lines, c)                    # the sweep's residual
    return time.perf_counter() - t0, float(lines) * n * n


def workload_config(n: int, k: int, c: float) -> dict:
    """The `config` of both arms' JSON lines (the same workload)."""
    return {"workload": f"q4_n{n}_expsine: Q^4, Ne={(n + 1) // k}/axis on [0,1]^3, n={n}, {n**3} DoF, "
                        "-Lap u + u = f, u = e^x sin(pi x) sin(pi y) sin(pi z), Dirichlet",
            "n": n, "k": k, "c": c, "dofs": n**3,
            "l2": "inputs larger than L2 (8 GB FP64 per array at n=999)"}


def oracle_cores() -> int:
    return int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args, rank: int, world: int):
    """The oracle as the reference arm: each step is one bounded slab sample of
    the n^3 refined solve, timed as it runs (no extrapolation): ms_per_step is
    the sample's wall time and value its DoF-equivalents per second."""
    if rank != 0:
        return 0
    n, k, c = args.n, 4, 1.0
    cores = oracle_cores()
    lines = args.reference_lines
    for _ in range(args.warmup):
        oracle_sample(n, k, c, lines)
    secs, units = [], 0.0
    for _ in range(args.steps):
        sec, u = oracle_sample(n, k, c, lines)
        secs.append(sec)
        units = u
    ms = float(np.mean(secs)) * 1e3
    value = units / (ms / 1e3) / 1e9
    sample = (f"oracle (numpy/BLAS FP64) refined solve restricted to {lines}-line slabs of the n={n} grid: "
              f"mode products along x, y, z (twice per fast solve, two fast solves) and one H-form apply, "
              f"{units:.4g} DoF-equivalents per step ({lines}/{n} of one solve)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(n, k, c), "dof_equivalents_per_step": units,
        "cpu_baseline": {"value": value, "unit": "GDoF/s", "cores": cores, "kind": "oracle", "sample": sample,
                         "seconds_per_step": ms / 1e3},
        "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------- our path

def single_gpu_only(gpus: int, world: int):
    """Reason to refuse a run on more than one GPU, else None.  The tcgen05
    mode-product kernels load the shared operand with TMA multicast inside
    thread-block clusters; their tensor maps cover this GPU's memory only, and
    the library is run one process on one GPU.  The solve does not shard
    (replicas only), so a multi-GPU run would add nothing."""
    if gpus != 1 or world != 1:
        return (f"single GPU only (--gpus {gpus}, WORLD_SIZE {world}): the tensor-core kernels use cluster TMA "
                "multicast and are run on one GPU per job")
    return None


def max_over_ranks(ms: float, dist, device: str) -> float:
    """The slowest rank's time (all ranks get it): the job's time for a weak-scaled
    replicated step.  device: "cuda" with NCCL, "cpu" with gloo."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput: the units all ranks processed / the job's time (per second)."""
    return units_per_rank * world / (ms / 1e3)


def timed(fn, steps, warmup, stream, torch, dist=None, before_stop=None):
    for _ in range(warmup):
        fn()
    if before_stop is not None:
        before_stop()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    if before_stop is not None:
        before_stop()  # the stream waits for work issued on other streams (the copies)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    if dist is not None:
        ms = max_over_ranks(ms, dist, "cuda")
        dist.barrier()
    return ms


def run_ours(args, rank: int, world: int, local_rank: int):
    import torch
    from paper_2310_00226_gb300 import sem3d
    from paper_2310_00226_gb300.inputs import exp_sine

    dist = None  # one GPU only: main() refuses more (see single_gpu_only)
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    peaks, peak_src = load_peaks()
    n, k, c = args.n, 4, 1.0
    dofs = n**3
    t_setup = time.perf_counter()
    plan = sem3d.Plan(n, n, n, k, (1.0, 1.0, 1.0), c)
    t_setup = time.perf_counter() - t_setup
    x = plan.nodes(0)
    u_ex_h, f_h = exp_sine(x, x, x, c)
    f = torch.from_numpy(f_h).cuda()
    u = torch.empty_like(f)

    # ---- headline: BF16x3 + FP64 refinement sweeps
    if args.tc_config != "auto":  # pin the tensor-core kernel (else set_precision measures both)
        for ax in range(3):
            plan.set_tc_config(ax, int(args.tc_config))
    t_tune = time.perf_counter()
    plan.set_precision("bf16x3", args.sweeps)
    t_tune = time.perf_counter() - t_tune
    tc_variant = [plan.tc_config(ax) for ax in range(3)]
    plan.set_residual(args.residual)
    plan.set_exact_residual(args.exact_residual)
    exact_kind = plan.exact_residual_kind()
    step = lambda: plan.solve(f, u, stream)  # noqa: E731
    for _ in range(args.warmup):
        step()
    plan.sync_check(stream)
    clk = ClockSampler(local_rank)
    clk.start()
    launches0 = plan.launch_count()
    ms = timed(step, args.steps, 0, stream, torch, dist)
    launches = plan.launch_count() - launches0
    # Per-kernel device times come from a second timed region of the same K
    # steps in which the library records an event pair around every launch on
    # the launch's stream; the headline region above records none.
    plan.profile(True)
    ms_profiled = timed(step, args.steps, 0, stream, torch, dist)
    tc_n, tc_ms = plan.profile_read("tc_mode_product")
    per_pass = {}
    for key in ("tc_x", "tc_y", "tc_z", "tc_f64_out"):
        pn, pms = plan.profile_read(key)
        per_pass[key] = {"launches": pn, "avg_ms": pms / max(1, pn)}
    st_n, st_ms = plan.profile_read("stencil")
    sp_n, sp_ms = plan.profile_read("split")
    plan.profile(False)
    clocks = clk.stop()
    plan.sync_check(stream)
    u_bf = u.clone()

    # accuracy of the headline result
    u_ex = torch.from_numpy(u_ex_h).cuda()
    err_exact = float((u_bf - u_ex).abs().max() / u_ex.abs().max())
    del u_ex
    Au = torch.empty_like(f)
    plan.apply(u_bf, Au, stream)
    rel_res = float((f - Au).abs().max() / f.abs().max())
    del Au

    # ---- the same BF16x3 path with FP64 residuals in every sweep
    f64res = dfres = fmares = None
    if args.fp64_residual_steps > 0:
        # the headline schedule with the other arithmetic for the FP64-accurate residuals
        other = "fp64" if args.exact_residual == "fixed" else "fixed"
        plan.set_exact_residual(other)
        ms_e = timed(step, args.fp64_residual_steps, 1, stream, torch, dist)
        plan.sync_check(stream)
        fmares = {"exact_residual": plan.exact_residual_kind(), "ms_per_step": ms_e,
                  "value": job_throughput(dofs, world, ms_e) / 1e9, "unit": "GDoF/s",
                  "steps": args.fp64_residual_steps, "warmup": 1,
                  "rel_linf_vs_headline": float((u - u_bf).abs().max() / u_bf.abs().max())}
        plan.set_exact_residual(args.exact_residual)
        plan.set_residual("fp64")
        ms_r = timed(step, args.fp64_residual_steps, 1, stream, torch, dist)
        plan.sync_check(stream)
        f64res = {"ms_per_step": ms_r, "value": job_throughput(dofs, world, ms_r) / 1e9, "unit": "GDoF/s",
                  "steps": args.fp64_residual_steps, "warmup": 1,
                  "rel_linf_vs_mixed": float((u - u_bf).abs().max() / u_bf.abs().max())}
        # every residual in double-FP32 (not FP64 refinement; reported beside the headline)
        plan.set_residual("df")
        ms_d = timed(step, args.fp64_residual_steps, 1, stream, torch, dist)
        plan.sync_check(stream)
        u_ex = torch.from_numpy(u_ex_h).cuda()
        dfres = {"ms_per_step": ms_d, "value": job_throughput(dofs, world, ms_d) / 1e9, "unit": "GDoF/s",
                 "steps": args.fp64_residual_steps, "warmup": 1,
                 "rel_linf_vs_mixed": float((u - u_bf).abs().max() / u_bf.abs().max()),
                 "rel_linf_vs_exact_solution": float((u - u_ex).abs().max() / u_ex.abs().max())}
        del u_ex
        plan.set_residual(args.residual)

    # ---- plain FP64 DMMA path (+1 FP64 sweep)
    fp64 = None
    if args.fp64_steps > 0:
        plan.set_precision("fp64", 1)
        plan.profile(True)
        ms64 = timed(step, args.fp64_steps, args.fp64_warmup, stream, torch, dist)
        f64_n, f64_ms = plan.profile_read("f64_mode_product")
        plan.profile(False)
        plan.sync_check(stream)
        diff = float((u - u_bf).abs().max() / u.abs().max())
        fp64 = {"ms_per_step": ms64, "value": job_throughput(dofs, world, ms64) / 1e9, "unit": "GDoF/s",
                "steps": args.fp64_steps, "warmup": args.fp64_warmup, "path": "FP64 DMMA mode products + 1 FP64 sweep",
                "rel_linf_bf16x3_vs_fp64": diff, "speedup_bf16x3_over_fp64": ms64 / ms,
                "dmma_kernel_avg_ms": f64_ms / max(1, f64_n),
                "dmma_achieved_tflops": 2.0 * n**4 / (f64_ms / max(1, f64_n) / 1e3) / 1e12}
        plan.set_precision("bf16x3", args.sweeps)

    # ---- FP32 CUDA-core tier (autotuned tiles) with FP64 refinement sweeps
    fp32 = None
    if args.fp32_steps > 0:
        u_ex = torch.from_numpy(u_ex_h).cuda()
        t0 = time.perf_counter()
        plan.set_precision("fp32", args.fp32_sweeps)  # runs the autotuner for new pass shapes
        tune_s = time.perf_counter() - t0
        plan.profile(True)
        ms_f = timed(step, args.fp32_steps, 1, stream, torch, dist)
        f_n, f_ms = plan.profile_read("f32_mode_product")
        plan.profile(False)
        plan.sync_check(stream)
        fp32 = {"path": "FP32 FFMA mode products (autotuned tiles) + FP64 refinement", "sweeps": args.fp32_sweeps,
                "steps": args.fp32_steps, "warmup": 1, "ms_per_step": ms_f,
                "value": job_throughput(dofs, world, ms_f) / 1e9, "unit": "GDoF/s", "autotune_s": tune_s,
                "rel_linf_vs_exact_solution": float((u - u_ex).abs().max() / u_ex.abs().max()),
                "rel_linf_vs_bf16x3": float((u - u_bf).abs().max() / u_bf.abs().max()),
                "pass_avg_ms": f_ms / max(1, f_n),
                "pass_tflops": 2.0 * n**4 / (f_ms / max(1, f_n) / 1e3) / 1e12,
                "tiles": [plan.tuned_config(a) for a in range(3)]}
        del u_ex
        plan.set_precision("bf16x3", args.sweeps)

    # ---- TF32 tensor-core tier (the single-precision arithmetic of Table 10):
    # bare (0 sweeps) and with FP64 refinement sweeps
    tf32 = None
    if args.tf32_steps > 0:
        u_ex = torch.from_numpy(u_ex_h).cuda()
        # TF32 dense peak: cuBLAS TF32 measured on this GPU (sustained loop, profiles/library_gemm_peaks.json),
        # else the measured sustained bf16 peak x the nominal TF32 / bf16 ratio (1.1 / 2.25 PF/s)
        tf32_peak, tf32_src = None, None
        try:
            with open(os.path.join(ROOT, "profiles", "library_gemm_peaks.json")) as fh:
                tf32_peak = float(json.load(fh)["tf32"]["sustained"])
            tf32_src = "cuBLAS TF32 GEMM, sustained, measured on GB300 (profiles/library_gemm_peaks.json)"
        except (OSError, ValueError, KeyError):
            tf32_peak = float(peaks.get("bf16_tflops_sustained", PEAKS_FALLBACK["bf16_tflops_sustained"])) * 1.1 / 2.25
            tf32_src = f"{peak_src} bf16_tflops_sustained x 1.1/2.25 (nominal TF32/bf16 ratio)"
        tf32 = {"path": "tcgen05 kind::tf32 mode products (rotating K-major layouts)", "steps": args.tf32_steps,
                "warmup": 1, "tf32_peak_tflops": tf32_peak, "tf32_peak_source": tf32_src}
        for label, sw in (("bare", 0), ("refined", args.tf32_sweeps)):
            plan.set_precision("tf32", sw)
            plan.profile(True)
            ms_t = timed(step, args.tf32_steps, 1, stream, torch, dist)
            t_n, t_ms = plan.profile_read("tc_mode_product")
            plan.profile(False)
            plan.sync_check(stream)
            tf32[label] = {"sweeps": sw, "ms_per_step": ms_t, "value": job_throughput(dofs, world, ms_t) / 1e9,
                           "unit": "GDoF/s", "rel_linf_vs_exact_solution":
                           float((u - u_ex).abs().max() / u_ex.abs().max()),
                           "tc_avg_ms": t_ms / max(1, t_n),
                           "tc_tflops": 2.0 * n**4 / (t_ms / max(1, t_n) / 1e3) / 1e12}
            tf32[label]["tc_frac_of_tf32_peak"] = tf32[label]["tc_tflops"] / tf32_peak
        del u_ex
        plan.set_precision("bf16x3", args.sweeps)

    # ---- end to end through the public API with host buffers
    e2e = None
    if args.e2e:
        f_pin = torch.from_numpy(f_h).pin_memory()
        u_pin = torch.empty(f_h.shape, dtype=torch.float64).pin_memory()

        # sem3d_solve_host: per call an 8-byte-per-DoF copy in, the solve, a copy out;
        # consecutive calls overlap one call's copies with another's solve.
        def e2e_step():
            plan.solve_host(f_pin, u_pin, stream)

        def e2e_wait():
            plan.solve_host_wait(stream)

        ms_e2e = timed(e2e_step, args.steps, args.warmup, stream, torch, dist, before_stop=e2e_wait)
        e2e = {"value": job_throughput(dofs, world, ms_e2e) / 1e9, "unit": "GDoF/s", "ms_per_step": ms_e2e,
               "h2d_bytes_per_step": int(f_pin.numel() * 8), "d2h_bytes_per_step": int(u_pin.numel() * 8)}
        del f_pin, u_pin

    # ---- roofline of the dominant kernel (tcgen05 BF16x3 mode product)
    tc_avg_ms = tc_ms / max(1, tc_n)
    flops_per_launch = 3 * 2.0 * n**4  # 3 bf16 products per useful FMA, 2 flops each, n^4 FMA per pass
    achieved = flops_per_launch / (tc_avg_ms / 1e3) / 1e12
    peak = float(peaks.get("bf16_tflops_sustained", PEAKS_FALLBACK["bf16_tflops_sustained"]))
    roofline = {"kernel": "mode_product_bf16x3 (tcgen05)", "bound": "tensor", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": tc_traffic_per_launch(n),
                "traffic_source": "profiles/roofline_inputs.json (ncu at n=511, scaled by DoF per launch)",
                "algorithmic_bytes_per_launch": 8.0 * ((n + 15) // 16 * 16) * n * n,
                "peak_source": f"{peak_src} bf16_tflops_sustained",
                "flops_per_launch": flops_per_launch, "avg_launch_ms": tc_avg_ms, "launches": tc_n,
                "share_of_step": tc_ms / (ms_profiled * args.steps),
                "kernel_times_from": (f"second timed region of {args.steps} steps with an event pair per launch "
                                      f"({ms_profiled:.2f} ms per step there; headline region {ms:.2f} ms)")}
    # The same fraction per unit of SM clock: the bench's median clock under load
    # against the clock the peak was measured at (a power-capped GEMM runs slower
    # clocks than a kernel that keeps the tensor pipe less busy).
    peak_mhz = (peaks.get("clocks_under_load") or {}).get("sm_mhz_median")
    if clocks.get("sm_mhz") and peak_mhz:
        a_ghz, p_ghz = achieved / (clocks["sm_mhz"] / 1e3), peak / (peak_mhz / 1e3)
        roofline["clock_normalised"] = {
            "achieved_tflops_per_ghz": a_ghz, "peak_tflops_per_ghz": p_ghz, "frac": a_ghz / p_ghz,
            "bench_sm_mhz_median": clocks["sm_mhz"], "peak_sm_mhz_median": peak_mhz,
            "frac_of_nominal_dense_rate": achieved / (152 * 8192 * clocks["sm_mhz"] * 1e6 / 1e12),
            "nominal_dense_rate": "8192 bf16 flop per clock per SM x 152 SMs x the bench's median SM clock"}
    kernels = {"tc_mode_product": {"launches": tc_n, "avg_ms": tc_avg_ms, "per_pass": per_pass},
               "residuals": {"launches": st_n, "ms_per_step": st_ms / max(1, args.steps),
                             "note": "every residual kernel of a step (double-FP32 sweeps, the FP64-accurate "
                                     "sweep and its scale reductions / conversion)"},
               "split": {"launches": sp_n, "avg_ms": sp_ms / max(1, sp_n),
                         "gbs": 12.0 * dofs / (sp_ms / max(1, sp_n) / 1e3) / 1e9}}

    cpu = None
    if rank == 0 and world == 1 and args.cpu_baseline:
        sec, units = oracle_sample(n, k, c, args.oracle_lines)
        cpu = {"value": units / sec / 1e9, "unit": "GDoF/s", "cores": oracle_cores(), "kind": "oracle",
               "seconds": sec, "dof_equivalents": units,
               "sample": (f"oracle refined solve restricted to {args.oracle_lines}-line slabs of the n={n} grid "
                          f"(mode products along x, y, z and one H-form apply; {args.oracle_lines}/{n} of a "
                          f"solve, {units:.4g} DoF-equivalents, {sec:.1f} s)")}

    line = {
        "metric": METRIC, "value": job_throughput(dofs, world, ms) / 1e9, "unit": "GDoF/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3 (fp32 accumulate) + f64 refinement", "data": "synthetic",
        "config": workload_config(n, k, c),
        "path": (f"tcgen05 BF16x3 mode products + {args.sweeps} refinement sweeps; residuals: "
                 + ("double-FP32 except the last" if args.residual == "mixed" else args.residual)
                 + f"; FP64-accurate residuals in {'64-bit integer fixed point' if exact_kind == 'fixed' else 'FP64 FMAs'}"),
        "parallelism": "single GPU", "setup_s": t_setup,
        "tc_kernel": {"per_axis": tc_variant, "legend": "0 = one CTA per 128x256 tile (W multicast in clusters of 4), "
                      "1 = cta_group::2 CTA pair per 256x256 tile", "chosen_by": "autotuner" if args.tc_config == "auto"
                      else "pinned", "set_precision_s": t_tune},
        "accuracy": {"rel_linf_vs_exact_solution": err_exact, "rel_residual_linf": rel_res},
        "roofline": roofline, "kernels": kernels, "gpu_launches": launches, "clocks": clocks,
        "fp64_path": fp64, "fp32_path": fp32, "tf32_path": tf32, "bf16x3_fp64_residuals": f64res, "bf16x3_other_exact_residual": fmares, "bf16x3_df_residuals": dfres, "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------- library GEMM peaks

def probe_peaks(args):
    """Dense GEMM rates of the vendor library on this GPU, as roofline
    denominators for the tiers whose dtype MEASURED_PEAKS.json does not cover:
    cuBLAS TF32 (torch.matmul on float32 with TF32 enabled), INT8 with INT32
    accumulation (torch._int_mm), FP64 and, for reference, bf16.  Each is
    timed with CUDA events as the best of 10 single calls (burst) and as the
    mean over a ~2 s back-to-back loop (sustained), with nvidia-smi clocks
    sampled during the loop.  Prints one JSON line."""
    import torch
    torch.cuda.set_device(0)
    dev = "cuda"
    res = {"probe": "library GEMM peaks", "n_gpus": 1, "gpu": torch.cuda.get_device_name(0)}

    def run(label, make, mm, flops):
        try:
            a, b = make()
            for _ in range(3):
                mm(a, b)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(10):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                mm(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            reps = max(3, int(2000.0 / best))
            clk = ClockSampler(0)
            clk.start()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                mm(a, b)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            clocks = clk.stop()
            res[label] = {"burst_tflops": flops / best / 1e9, "sustained_tflops": flops / ms / 1e9,
                          "burst_ms": best, "sustained_ms": ms, "reps": reps, "clocks": clocks}
        except Exception as exc:  # noqa: BLE001 - reported, not hidden
            res[label] = {"error": f"{type(exc).__name__}: {exc}"}
        torch.cuda.empty_cache()

    n = 8192
    torch.backends.cuda.matmul.allow_tf32 = True
    run("tf32", lambda: (torch.randn(n, n, device=dev), torch.randn(n, n, device=dev)), torch.matmul, 2.0 * n**3)
    torch.backends.cuda.matmul.allow_tf32 = False
    run("bf16", lambda: (torch.randn(n, n, device=dev, dtype=torch.bfloat16),
                         torch.randn(n, n, device=dev, dtype=torch.bfloat16)), torch.matmul, 2.0 * n**3)
    run("int8", lambda: (torch.randint(-128, 127, (n, n), device=dev, dtype=torch.int8),
                         torch.randint(-128, 127, (n, n), device=dev, dtype=torch.int8)),
        torch._int_mm, 2.0 * n**3)
    m = 4096
    run("fp64", lambda: (torch.randn(m, m, device=dev, dtype=torch.float64),
                         torch.randn(m, m, device=dev, dtype=torch.float64)), torch.matmul, 2.0 * m**3)
    res["unit"] = "TFLOP/s (TOP/s for int8)"
    print(json.dumps(res), flush=True)
    return 0


# --------------------------------------------------------------------- other workloads

def _timed_host(fn, steps, warmup, torch):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) * 1e3 / steps


def _progress(msg: str):
    print(f"bench.py [{time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def run_workload(args, rank: int):
    """Batched Helmholtz, Cahn-Hilliard and Schroedinger-PCG workloads (one JSON
    line each; not the headline metric)."""
    import torch
    from paper_2310_00226_gb300 import sem3d
    from paper_2310_00226_gb300.inputs import batched_helmholtz, harmonic_potential, random_rhs
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    line = {"workload": args.workload, "n_gpus": 1, "data": "synthetic", "higher_is_better": True}
    if args.workload == "batched":
        probs = batched_helmholtz(args.batch_count)
        plans, fs, us = [], [], []
        for pr in probs:
            p = sem3d.Plan(*pr["n3"], pr["k"], (1.0, 1.0, 1.0), pr["c"])
            plans.append(p)
            nx, ny, nz = pr["n3"]
            fs.append(torch.from_numpy(random_rhs(nx, ny, nz, pr["seed"])).cuda())
            us.append(torch.empty_like(fs[-1]))
        dofs = sum(p.numel for p in plans)
        _progress(f"batched: {len(plans)} plans, {dofs} DoF")
        res = {}
        for prec, sweeps in (("fp32", 2), ("bf16x3", 3)):
            for p in plans:
                p.set_precision(prec, sweeps)
            _progress(f"batched: {prec} set_precision done")
            ms = _timed_host(lambda: sem3d.solve_batched(plans, fs, us, stream), args.steps, args.warmup, torch)
            plans[0].sync_check(stream)
            _progress(f"batched: {prec} grouped {ms:.1f} ms per batch")
            res[prec] = {"ms_per_batch": ms, "GDoF_per_s": dofs / (ms / 1e3) / 1e9, "sweeps": sweeps,
                         "path": ("grouped FP32 launch per pass" if prec == "fp32" else
                                  "grouped tcgen05 CTA-pair launch per pass (tile queue over all problems)")}
        # the same BF16x3 solves as one sem3d_solve call per plan, one after another on the stream, for comparison
        def per_plan():
            for q, p in enumerate(plans):
                p.solve(fs[q], us[q], stream)

        ms = _timed_host(per_plan, args.steps, args.warmup, torch)
        plans[0].sync_check(stream)
        res["bf16x3_per_plan"] = {"ms_per_batch": ms, "GDoF_per_s": dofs / (ms / 1e3) / 1e9, "sweeps": 3,
                                  "path": "each plan's sem3d_solve in turn on one stream (no grouping)"}
        _progress(f"batched: per-plan solves {ms:.1f} ms per batch")
        line.update({"metric": f"{args.batch_count} batched Helmholtz solves (uneven n in {{63..511}}, k in {{2,3,4,6}}): GDoF/s",
                     "value": res["bf16x3"]["GDoF_per_s"], "unit": "GDoF/s", "total_dofs": dofs, "tiers": res,
                     "steps": args.steps, "warmup": args.warmup})
    elif args.workload == "ch":
        n, k = args.workload_n or 511, 2
        p = sem3d.Plan(n, n, n, k, (2 * np.pi,) * 3, 0.0)
        rng = np.random.Generator(np.random.PCG64(20231001))
        phi0 = torch.from_numpy(rng.uniform(-0.05, 0.05, (n, n, n))).cuda()
        res = {}
        tiers = ["bf16x3", "fp32"] + (["fp64"] if args.ch_fp64_steps > 0 else [])
        for prec in tiers:
            p.set_precision(prec, 0)
            steps = {"bf16x3": args.ch_steps, "fp32": max(1, args.ch_steps // 10), "fp64": args.ch_fp64_steps}[prec]
            pm, pn = phi0.clone(), phi0.clone()
            p.ch_run(pm, pn, 3, 0.05, 1.0, 1e-4, 2.0, stream)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p.ch_run(pm, pn, steps, 0.05, 1.0, 1e-4, 2.0, stream)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3 / steps
            p.sync_check(stream)
            res[prec] = {"ms_per_step": ms, "steps": steps, "max_abs_phi": float(pn.abs().max())}
        line.update({"metric": f"Cahn-Hilliard BDF2 step, Q^2 n={n} on [0,2pi]^3 ({n**3:.3g} DoF): ms/step",
                     "value": res["bf16x3"]["ms_per_step"], "unit": "ms/step", "higher_is_better": False,
                     "tiers": res, "params": {"eps": 0.05, "m": 1.0, "dt": 1e-4, "S": 2.0}})
    elif args.workload == "pcg":
        n, k = args.workload_n or 1023, 4
        p = sem3d.Plan(n, n, n, k, (1.0, 1.0, 1.0), 25.0)
        x = p.nodes(0)
        V = torch.from_numpy(harmonic_potential(x, x, x, 100.0)).cuda()
        f = torch.ones_like(V)
        u = torch.empty_like(V)
        res = {}
        variants = [("bf16x3", 0), ("bf16x3", 1)] + ([("fp64", 0)] if args.pcg_fp64 else [])
        for prec, sweeps in variants:
            p.set_precision(prec, sweeps)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, rr = p.pcg(V, f, u, rtol=1e-10, maxit=200, stream=stream)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3
            res[f"{prec}_sweeps{sweeps}"] = {"ms": ms, "iterations": it, "relres": rr, "ms_per_iteration": ms / it,
                                             "u_max": float(u.abs().max())}
        line.update({"metric": f"Schroedinger -Lap u + 100|x-1/2|^2 u = 1, Q^4 n={n} ({n**3:.3g} DoF), PCG to 1e-10: s",
                     "value": min(r["ms"] for r in res.values()) / 1e3, "unit": "s", "higher_is_better": False,
                     "preconditioner": res})
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1, help="must be 1: the library runs on one GPU")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=999, help="interior nodes per axis (n+1 divisible by 4)")
    ap.add_argument("--sweeps", type=int, default=3)
    ap.add_argument("--residual", choices=["mixed", "fp64", "df"], default="mixed")
    ap.add_argument("--exact-residual", choices=["fixed", "fp64"], default="fixed",
                    help="arithmetic of the FP64-accurate refinement residuals (64-bit fixed point or FP64 FMAs)")
    ap.add_argument("--fp64-residual-steps", type=int, default=3,
                    help="also time the BF16x3 path with FP64 residuals in every sweep (0 = skip)")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--fp32-steps", type=int, default=2,
                    help="timed solves of the FP32 CUDA-core tier with --fp32-sweeps sweeps; 0 skips it")
    ap.add_argument("--fp32-sweeps", type=int, default=2)
    ap.add_argument("--tf32-steps", type=int, default=5,
                    help="timed solves of the TF32 tier (bare, and refined with --tf32-sweeps); 0 skips it")
    ap.add_argument("--tf32-sweeps", type=int, default=7)
    ap.add_argument("--fp64-warmup", type=int, default=1)
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--oracle-lines", type=int, default=191,
                    help="slab thickness of the oracle CPU-baseline sample (~20 s on 16 cores); (lines+1) %% 4 == 0")
    ap.add_argument("--reference-lines", type=int, default=31,
                    help="slab thickness of each step of --impl reference (~5 s per step on 16 cores)")
    ap.add_argument("--tc-config", choices=["auto", "0", "1"], default="auto",
                    help="tensor-core kernel of the headline: autotuned, 0 = one CTA per tile, 1 = CTA pair")
    ap.add_argument("--probe-peaks", action="store_true",
                    help="time the vendor library's TF32, bf16, INT8 and FP64 GEMMs (roofline denominators) and exit")
    ap.add_argument("--workload", choices=["solve", "batched", "ch", "pcg"], default="solve",
                    help="solve = the headline n=999 solve; the others time the batched, Cahn-Hilliard and PCG workloads")
    ap.add_argument("--ch-steps", type=int, default=1000)
    ap.add_argument("--workload-n", type=int, default=None,
                    help="grid size of the ch (default 511) or pcg (default 1023) workload, for small profiling runs")
    ap.add_argument("--batch-count", type=int, default=64, help="problems in the batched workload")
    ap.add_argument("--ch-fp64-steps", type=int, default=0,
                    help="also time this many Cahn-Hilliard steps in the FP64 tier (~1.2 s per step at n=511)")
    ap.add_argument("--pcg-fp64", action="store_true",
                    help="also run the PCG with the FP64 (DMMA) preconditioner (~13 s per iteration at n=1023)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.probe_peaks:
        return probe_peaks(args) if world == 1 else 2
    refusal = single_gpu_only(args.gpus, world)
    if refusal:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "n_gpus": max(args.gpus, world), "unavailable": refusal}), flush=True)
        print(f"bench.py: {refusal}", file=sys.stderr, flush=True)
        return 2
    if args.workload != "solve":
        return run_workload(args, rank)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
