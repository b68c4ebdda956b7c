"""Benchmark: ChFSI H.X applies/s on the 32-atom erf cluster (lmax 30, 48 radial functions,
d = 46128, 96 x 60 x 120 grid, 80 states, Chebyshev degree 16) on one GB300.

A step is one ChFSI iteration (Sec. 3.2.1) in its steady state, from Ritz vectors, their
H X and Ritz values (cs_chfsi_step_ritz):
  - the degree-16 Chebyshev filter in residual form: 15 H.X block products in the chosen
    precision on the deviation from X s_16(Theta), with the three-term recurrence fused into
    the H.X epilogue. The default is the mixed form: split-BF16 tensor-core radial
    contractions and phi transforms, FP32 Legendre sums;
  - Cholesky-QR (two passes);
  - Rayleigh-Ritz: one H.X, Gram, eigensolve, rotations and residual norms. By default the H.X
    and the Gram matrices and rotations run in double-float (FP64-class); the factorisation,
    eigensolve and residual norms run in FP64.
value = state-columns multiplied by H per second = (H.X products per step) * n_s / step time
(16 * 80 in residual form, 17 * 80 with --form plain), summed over ranks (each rank runs its
own block: weak scaling, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp32|fp64|df64]
                    [--form ritz|plain]
    python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "ChFSI H·X applies/s and SCF time to 1e-6 Ha: mixed/batched vs FP64, 1 GB300"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 / FP32 ALU peaks of one GB300: FP64 nominal 1.25 TFLOP/s; FP32 = 152 SMs x 128 lanes
# x 2 flop x 2.07 GHz (maximum SM clock).
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# double-float: one multiply-add (2 flops) costs 15 FP32 instructions (df64.cuh), so the
# FP32 issue rate bounds it at 2/15 of the FP32 multiply-add rate
DF64_PEAK_TFLOPS = FP32_PEAK_TFLOPS / 2 * 2 / 15


def _rank_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ------------------------------------------------------------------ multi-rank aggregation
def reduce_max_time(local_ms: float, world: int, device=None) -> float:
    """Max over ranks of a rank's timed milliseconds (the slowest rank sets the job time).
    Uses the process group only for timing; nothing of the data path crosses ranks."""
    if world <= 1:
        return float(local_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(applies_per_step_per_rank: float, world: int, ms_per_step: float) -> float:
    """Whole-job applies/s: every rank filters its own block (weak scaling)."""
    return world * applies_per_step_per_rank / (ms_per_step / 1e3)


def rank_block_seed(base_seed: int, rank: int) -> int:
    """Each rank draws its own state block (independent problems, no exchange)."""
    return base_seed + 1000 * rank


# ------------------------------------------------------------------ algorithmic work
def algorithmic_flops(w, n_s):
    """Per-state flop counts of one H.X (FFT count for phi, parity-folded Legendre)."""
    L, N, nr, nt, nph = w.L, w.nmax, w.n_r, w.n_theta, w.n_phi
    f_rad = 2.0 * nr * N * L * L                      # one direction
    f_leg = 2.0 * nt * L * L * nr / 2.0               # one direction, folded
    f_phi = 2.5 * nph * math.log2(nph) * nr * nt      # one direction (real FFT estimate)
    f_v = float(nr * nt * nph)
    return {"radial_synth": f_rad * n_s, "angular": (2 * f_leg + 2 * f_phi + f_v) * n_s,
            "radial_anal": f_rad * n_s,
            # the FP32-pipe share of the mixed angular kernel (its phi transforms run on tcgen05)
            "angular_fp32_pipe": (2 * f_leg + f_v) * n_s}


def dense_flops(d, n):
    # CholQR twice (Gram + rotation) + RR (Gram + two rotations)
    return 2 * (2.0 * d * n * n + 2.0 * d * n * n) + (2.0 * d * n * n + 4.0 * d * n * n)


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu --set full
# capture of the kernel as it stands, on this workload; a class without a capture reports null
NCU_TRAFFIC_BYTES = {"angular_f32": 32.496384e6 + 1024.0}  # k_angular_tc (mixed default)


# the profiling recipe's fallback denominators, used only when the generated peaks file
# is absent: one earlier GB300 measurement (HBM copy, cuBLAS bf16 burst and sustained)
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "source": "fallback"}


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        p.setdefault("source", "measured")
        return p
    except (OSError, ValueError):
        return dict(FALLBACK_PEAKS)


def peak_word(peaks):
    return "fallback" if peaks.get("source") == "fallback" else "measured"


def roofline_table(cs, w, d, n_s, prec, prof_ms, prof_n, steps, dense_prec):
    """Per kernel class: launches, share of device time, algorithmic TFLOP/s and the fraction
    of the pipe that bounds it; the dominant class becomes the `roofline` object. The dense
    class (Gram matrices and rotations of CholQR2 and Rayleigh-Ritz, factor, eigensolve) is
    rated against the pipe its Gram matrices and rotations run on: FP64, or the FP32 pipe in
    double-float."""
    from paper_1404_3773_gb300 import CS_DF64, CS_FP64_SLICED, CS_MIXED_BF16
    names = cs.profile_class_names()
    af = algorithmic_flops(w, n_s)
    peaks = measured_peaks()
    bf16 = peaks.get("bf16_tflops_sustained")
    total = max(1e-9, sum(prof_ms))
    classes = {}
    for i, name in enumerate(names):
        if prof_n[i] == 0:
            continue
        kind = "f32" if name.endswith("_f32") else ("df64" if name.endswith("_df64") else "f64")
        fam = name.rsplit("_", 1)[0] if kind != "f64" else name
        f32 = kind == "f32"
        per_ms = prof_ms[i] / prof_n[i]
        mixed_ang = f32 and prec == CS_MIXED_BF16 and fam == "angular"
        if mixed_ang:
            flops = af["angular_fp32_pipe"]
        elif fam in ("radial_synth", "radial_anal", "angular"):
            flops = af[fam]
        elif fam == "dense":
            flops = dense_flops(d, n_s) / max(1.0, prof_n[i] / steps)
        else:
            flops = None
        if f32 and prec == CS_MIXED_BF16 and fam.startswith("radial") and bf16:
            bound, peak, src = "tensor", bf16, f"{peak_word(peaks)} bf16 sustained"
        elif mixed_ang:
            bound, peak, src = "alu", FP32_PEAK_TFLOPS, (
                "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz; counted: the Legendre sums and W V "
                "on the FP32 pipe (the phi transforms run on tcgen05 and are not counted)")
        elif f32:
            bound, peak, src = "alu", FP32_PEAK_TFLOPS, "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"
        elif fam == "dense" and dense_prec == CS_FP64_SLICED and bf16:
            # each FP64 product is 36 BF16 slice products (8 digits, pairs k + l <= 7)
            bound, peak, src = "tensor", bf16 / 36.0, (
                f"{peak_word(peaks)} bf16 sustained / 36 (FP64-equivalent rate of the slice "
                "products; the class also holds the FP64 factor, eigensolve and residual kernels)")
        elif kind == "df64" or (fam == "dense" and dense_prec == CS_DF64):
            bound, peak, src = "alu", DF64_PEAK_TFLOPS, ("FP32 issue rate / 15 instructions "
                                                         "per double-float multiply-add")
        else:
            bound, peak, src = "alu", FP64_PEAK_TFLOPS, "FP64 nominal 1.25 TFLOP/s (GB300)"
        ach = flops / (per_ms / 1e3) / 1e12 if flops else None
        classes[name] = {"launches": int(prof_n[i]), "ms": round(prof_ms[i], 4),
                         "share": round(prof_ms[i] / total, 4),
                         "avg_launch_ms": round(per_ms, 5),
                         "flops_per_launch": flops,
                         "achieved": round(ach, 4) if ach else None,
                         "bound": bound, "peak": round(peak, 3), "unit": "TFLOP/s",
                         "frac": round(ach / peak, 4) if ach else None, "peak_source": src}
    # the dominant kernel: "dense" lumps many small kernels (Gram, GEMM, factor, eigensolve), so
    # the roofline object is taken over the classes that are one kernel each
    single = [k for k in classes if not k.startswith("dense")] or list(classes)
    dom = max(single, key=lambda k: classes[k]["ms"])
    c = classes[dom]
    roofline = {"bound": c["bound"], "kernel": dom, "achieved": c["achieved"], "peak": c["peak"],
                "unit": "TFLOP/s", "frac": c["frac"], "traffic": NCU_TRAFFIC_BYTES.get(dom),
                "peak_source": c["peak_source"], "flops_per_launch": c["flops_per_launch"],
                "avg_launch_ms": c["avg_launch_ms"], "share": c["share"]}
    return roofline, classes


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows),
                "power_w_max": max((float(r[3]) for r in self.rows
                                    if r[3].replace(".", "").isdigit()), default=None)}


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    rank, world, local = _rank_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    import paper_1404_3773_gb300 as cs
    from paper_1404_3773_gb300 import CS_FP32, CS_FP64, CS_MIXED_BF16

    from paper_1404_3773_gb300 import CS_DF64, CS_FP64_SLICED
    PREC = {"fp64": CS_FP64, "fp32": CS_FP32, "mixed": CS_MIXED_BF16, "df64": CS_DF64,
            "sliced": CS_FP64_SLICED}
    NAME = {v: k for k, v in PREC.items()}
    prec = PREC[args.precision]
    w = W.erf_cluster_32()
    n_s, degree = w.n_s, w.degree
    ctx = cs.cs_basis_init(w.R, w.lmax, w.nmax, w.n_r, w.n_theta, w.n_phi, 0, local)
    v = w.potential_at(cs.grid_points(ctx))
    cs.cs_set_potential(ctx, torch.tensor(v, dtype=torch.float64, device=dev))
    d = ctx.d
    # Rayleigh-Ritz projects an H X in the filter's precision ("same"), FP64 or double-float;
    # the Gram matrices and rotations run in FP64 or double-float
    rr_prec = prec if args.rr_precision == "same" else PREC[args.rr_precision]
    dense_prec = PREC[args.dense_precision]
    cs.cs_set_rr_precision(ctx, rr_prec)
    cs.cs_set_dense_precision(ctx, dense_prec)
    # each rank filters its own block of states (independent seeds)
    X0h = W.gaussian_block(rank_block_seed(w.x_seed, rank), d, n_s)
    X0 = torch.tensor(np.ascontiguousarray(X0h.T), device=dev)
    work = ctx.workspace(n_s, prec)
    theta = torch.empty(n_s, dtype=torch.float64, device=dev)
    resid = torch.empty_like(theta)
    # bounds (untimed set-up): Lanczos upper bound, first-pass interval, then one
    # iteration to reach the steady-state interval used by every timed step
    v0 = torch.tensor(W.gaussian(4242 + rank, d), device=dev)
    b, tmin = cs.cs_lanczos_bound(ctx, v0, 10, work)
    cs.cs_cholqr(ctx, X0, work)
    a0, a = tmin, tmin + (b - tmin) / 10.0
    Xs = X0.clone()
    cs.cs_chfsi_step(ctx, Xs, degree, a, b, a0, theta, resid, prec, work)
    th = theta.cpu().numpy()
    a, a0 = float(th[-1]), float(th[0])
    X0.copy_(Xs)
    # H X and Ritz values of the starting Ritz vectors (the residual form's inputs, which a
    # ChFSI loop carries from one iteration to the next)
    HX0 = torch.empty_like(X0)
    cs.cs_rayleigh_ritz(ctx, X0, theta, resid, HX0, work)
    th0 = theta.clone()
    X = torch.empty_like(X0)
    HX = torch.empty_like(X0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2
    ritz = args.form == "ritz"
    hx_per_step = degree if ritz else degree + 1  # filter products + the Rayleigh-Ritz one

    def reset():
        X.copy_(X0)
        if ritz:
            HX.copy_(HX0)
            theta.copy_(th0)

    def step():
        if ritz:
            cs.cs_chfsi_step_ritz(ctx, X, HX, degree, a, b, a0, theta, resid, prec, work)
        else:
            cs.cs_chfsi_step(ctx, X, degree, a, b, a0, theta, resid, prec, work)

    for _ in range(args.warmup):
        reset()
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
        time.sleep(0.5)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    n_launch0 = cs.cs_launch_count(ctx)
    cs.cs_profile_begin(ctx)
    total_ms = 0.0
    launches_timed = 0
    for _ in range(args.steps):
        reset()
        flush.fill_(1.0)  # L2 flush between timed iterations (not timed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        before = cs.cs_launch_count(ctx)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        launches_timed += cs.cs_launch_count(ctx) - before
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    prof_ms, prof_n = cs.cs_profile_end(ctx)
    if world > 1:
        total_ms = reduce_max_time(total_ms, world, device=dev)
        torch.distributed.barrier()
    if rank == 0:
        time.sleep(0.3)
        clocks.stop()
    ms_per_step = total_ms / args.steps
    applies_per_step = hx_per_step * n_s
    value = job_value(applies_per_step, world, ms_per_step)

    # ---- end to end through the public API: host (pinned) inputs in (the block, and in
    # residual form its H X and Ritz values), Ritz vectors + values (and their H X) out
    Xh = X0.cpu().pin_memory()
    HXh = HX0.cpu().pin_memory()
    thh_in = th0.cpu().pin_memory()
    Xout = torch.empty_like(Xh).pin_memory()
    HXout = torch.empty_like(Xh).pin_memory()
    thh = torch.empty(n_s, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        X.copy_(Xh, non_blocking=True)
        if ritz:
            HX.copy_(HXh, non_blocking=True)
            theta.copy_(thh_in, non_blocking=True)
        step()
        Xout.copy_(X, non_blocking=True)
        thh.copy_(theta, non_blocking=True)
        if ritz:
            HXout.copy_(HX, non_blocking=True)
    e1.record(stream)
    e1.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    nblk = 2 if ritz else 1
    h2d = nblk * X0.numel() * 8 + (n_s * 8 if ritz else 0)
    d2h = nblk * X0.numel() * 8 + n_s * 8

    # ---- Ritz values of one step from X0 with the reduced Rayleigh-Ritz apply against the
    # same step with an FP64 apply (wanted states), and the other precisions' step times
    def one_step(p_filter, p_rr, p_dense=None):
        cs.cs_set_rr_precision(ctx, p_rr)
        cs.cs_set_dense_precision(ctx, dense_prec if p_dense is None else p_dense)
        wk = ctx.workspace(n_s, p_filter)
        X.copy_(X0)
        cs.cs_chfsi_step(ctx, X, degree, a, b, a0, theta, resid, p_filter, wk)
        return theta.cpu().numpy().copy(), wk

    th_red, _ = one_step(prec, rr_prec)
    th_64, _ = one_step(prec, CS_FP64, CS_FP64)
    ritz_dev = float(np.max(np.abs(th_red[:w.n_want] - th_64[:w.n_want])))

    def time_variant(p_filter, p_rr, p_dense, form, reps=3):
        one_step(p_filter, p_rr, p_dense)  # warm (tables, workspace)
        wk = ctx.workspace(n_s, p_filter)
        # the residual form's inputs: H X of X0 in this Rayleigh-Ritz precision
        Xr, HXr = X0.clone(), torch.empty_like(X0)
        cs.cs_rayleigh_ritz(ctx, Xr, theta, resid, HXr, wk)
        thr = theta.clone()

        def run():
            X.copy_(Xr)
            if form == "ritz":
                HX.copy_(HXr)
                theta.copy_(thr)
                cs.cs_chfsi_step_ritz(ctx, X, HX, degree, a, b, a0, theta, resid, p_filter, wk)
            else:
                cs.cs_chfsi_step(ctx, X, degree, a, b, a0, theta, resid, p_filter, wk)

        for _ in range(2):
            run()
        tot = 0.0
        for _ in range(reps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            # the block copies sit inside this interval (two device block copies, ~20 us)
            e0.record(stream)
            run()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        ms = tot / reps
        nhx = degree if form == "ritz" else degree + 1
        return {"ms_per_step": round(ms, 4), "form": form, "hx_per_step": nhx,
                "value": round(nhx * n_s / (ms / 1e3), 2)}

    variants = None
    if not args.no_variants:
        variants = {}
        for name, pf, prr, pd, form in (
                ("fp64", CS_FP64, CS_FP64, CS_FP64, "plain"),
                ("df64", CS_DF64, CS_DF64, CS_DF64, "plain"),
                ("fp32_rr_fp64", CS_FP32, CS_FP64, CS_FP64, "plain"),
                ("fp32_rr_df64", CS_FP32, CS_DF64, CS_DF64, "plain"),
                ("mixed_rr_df64", CS_MIXED_BF16, CS_DF64, CS_DF64, "plain"),
                ("mixed_rr_fp64", CS_MIXED_BF16, CS_FP64, CS_FP64, "plain"),
                ("fp64_ritz", CS_FP64, CS_FP64, CS_FP64, "ritz"),
                ("fp32_ritz_rr_df64", CS_FP32, CS_DF64, CS_DF64, "ritz"),
                ("mixed_ritz_rr_df64", CS_MIXED_BF16, CS_DF64, CS_DF64, "ritz"),
                ("mixed_ritz_rr_fp64", CS_MIXED_BF16, CS_FP64, CS_FP64, "ritz"),
                ("mixed_ritz_rr_df64_sliced", CS_MIXED_BF16, CS_DF64, CS_FP64_SLICED, "ritz"),
                ("mixed_ritz_rr_fp64_sliced", CS_MIXED_BF16, CS_FP64, CS_FP64_SLICED,
                 "ritz")):
            v = time_variant(pf, prr, pd, form)
            v.update({"filter": NAME[pf], "rayleigh_ritz_apply": NAME[prr],
                      "gram_and_rotations": NAME[pd]})
            variants[name] = v
    cs.cs_set_rr_precision(ctx, rr_prec)
    cs.cs_set_dense_precision(ctx, dense_prec)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- roofline of the dominant kernel class (device time measured live above)
    roofline, classes = roofline_table(cs, w, d, n_s, prec, prof_ms, prof_n, args.steps,
                                       dense_prec)
    # the FP32 / FP64 FMA rates measured on this device, beside the nominal unit-count peaks
    alu = None
    try:
        f32, f64 = cs.cs_measure_peaks(local)
        alu = {"fp32_tflops": round(f32, 2), "fp64_tflops": round(f64, 3),
               "fp32_nominal_tflops": round(FP32_PEAK_TFLOPS, 2),
               "fp64_nominal_tflops": FP64_PEAK_TFLOPS,
               "how": "8 independent FMA chains per thread, 4 x 256 threads per SM, best of 5"}
        if roofline.get("bound") == "alu" and roofline.get("achieved") and f32 > 0 and \
                roofline.get("peak") == round(FP32_PEAK_TFLOPS, 3):
            roofline["frac_of_measured_fp32"] = round(roofline["achieved"] / f32, 4)
    except Exception as exc:  # the measurement is context, not the result
        alu = {"error": str(exc)}

    step_times = step_breakdown(classes, args.steps, hx_per_step - 1, ms_per_step, prec,
                                rr_prec)

    batched = None if args.no_batched else batched_measure(dev)
    at_scale = None if args.no_at_scale else at_scale_measure(dev)
    at_scale_chfsi = None if args.no_at_scale_chfsi else at_scale_chfsi_measure(dev)
    scf = None if args.no_scf else scf_measure(dev)
    first_solve = None if args.no_scf else first_solve_measure(dev)
    eigen_gate = None if args.no_scf else eigen_gate_measure(dev)
    learned_init = None if args.no_scf else learned_init_measure(dev)
    cpu = cpu_baseline(w, budget_s=args.cpu_seconds) if not args.no_cpu_baseline else None
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "applies/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32+f64", "mixed": "bf16x3+f32+f64",
                  "df64": "df64+f64"}[args.precision],
        "data": "synthetic (seeded erf pseudo-atom cluster and Gaussian state block)",
        "config": {"workload": "erf32_l30_n48: 32 erf atoms in r<=8, R=14, lmax=30, 48 radial "
                               "fns/l, d=46128, grid 96x60x120, 80 states, degree 16",
                   "step": ("one steady-state ChFSI iteration: residual-form filter (15 H.X on "
                            "the deviation) + CholQR x2 + Rayleigh-Ritz (1 H.X in the "
                            "rayleigh_ritz_apply precision)") if ritz else
                           ("one ChFSI iteration: filter (16 H.X) + CholQR x2 + Rayleigh-Ritz "
                            "(1 H.X in the rayleigh_ritz_apply precision)"),
                   "filter_form": args.form,
                   "hx_per_step": hx_per_step,
                   "filter_precision": args.precision,
                   "rayleigh_ritz_apply": NAME[rr_prec],
                   "gram_and_rotations": NAME[dense_prec],
                   "factorisation_eigensolve_residuals": "fp64",
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"replicas x{world} (independent state blocks)"},
        "roofline": roofline,
        "kernel_classes": classes,
        "step_times": step_times,
        "cpu_baseline": cpu,
        "e2e": {"value": round(world * applies_per_step / (e2e_ms / 1e3), 2),
                "unit": "applies/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches_timed),
        "batched": batched,
        "at_scale": at_scale,
        "at_scale_chfsi": at_scale_chfsi,
        "scf": scf,
        "first_solve": first_solve,
        "eigen_gate": eigen_gate,
        "learned_init": learned_init,
        "clocks": clocks.summary(),
        "ritz": {"theta_min": float(th_red[0]), "max_dev_wanted_vs_fp64_rr": ritz_dev,
                 "n_wanted": w.n_want},
        "variants": variants,
        "alu_peaks": alu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def step_breakdown(classes, steps, degree, ms_per_step, prec, rr_prec):
    """Per ChFSI iteration: the filter pass (degree H.X with the recurrence), one Chebyshev
    step, the Rayleigh-Ritz H.X and the dense part, from the per-class device times; and the
    step's roofline time, the sum over classes of algorithmic flops / the bounding pipe's peak
    (every class here is ALU-bound: its bytes / HBM bandwidth is far smaller)."""
    from paper_1404_3773_gb300 import CS_FP64, CS_FP32, CS_MIXED_BF16, CS_DF64
    sfx = {CS_FP64: "", CS_FP32: "_f32", CS_MIXED_BF16: "_f32", CS_DF64: "_df64"}
    fams = ("radial_synth", "angular", "radial_anal", "kb")

    def hx_ms(suffix):
        return sum(classes[f + suffix]["ms"] for f in fams if f + suffix in classes) / steps

    filt = hx_ms(sfx[prec])
    if sfx[rr_prec] == sfx[prec]:  # filter and Rayleigh-Ritz applies share the classes
        rr = filt / (degree + 1)
        filt -= rr
    else:
        rr = hx_ms(sfx[rr_prec])
    dense = classes["dense"]["ms"] / steps if "dense" in classes else 0.0
    roof = 0.0
    for c in classes.values():
        if c["flops_per_launch"]:
            roof += c["launches"] / steps * c["flops_per_launch"] / (c["peak"] * 1e12) * 1e3
    return {"filter_pass_ms": round(filt, 4), "cheb_step_ms": round(filt / degree, 4),
            "rayleigh_ritz_apply_ms": round(rr, 4), "dense_ms": round(dense, 4),
            "step_ms": round(ms_per_step, 4),
            "roofline_ms": round(roof, 4), "roofline_frac": round(roof / ms_per_step, 4)}


def scf_measure(dev, precisions=("mixed", "fp32", "fp64"), tol=1e-6, max_iter=80):
    """SCF time to |dE| <= tol Ha on the 32-atom cluster (Z = 4 erf pseudo-atoms, 128
    electrons, 80 states, degree 16): Gaussian starting density (sigma 1 bohr per atom),
    Fermi-Dirac kT = 6.3e-4 Ha (200 K), Anderson mixing of the effective potential (beta 0.3,
    history 8), ChFSI to a 1e-3 residual in the first iteration, then one ChFSI iteration per
    SCF iteration. Wall clock around the whole loop (every SCF step synchronises)."""
    import torch

    import paper_1404_3773_gb300 as cs
    from workloads.device import erf_cluster_potential_t, gaussian_atom_density_t
    w = W.erf_cluster_32()
    atoms = w.atoms()
    Z = w.extra["Z"]
    e_ion = sum(Z * Z / float(np.linalg.norm(atoms[i] - atoms[j]))
                for i in range(len(atoms)) for j in range(i))
    idx = torch.device(dev).index or 0
    out = {"workload": "erf32_l30_n48 SCF: 32 Z=4 erf pseudo-atoms, 128 electrons, 80 states, "
                       "degree 16, kT 200 K, Anderson beta 0.3 / history 8, "
                       f"stop at |dE| <= {tol:g} Ha (total)",
           "e_ion": e_ion}
    for name in precisions:
        prec = {"fp32": cs.CS_FP32, "fp64": cs.CS_FP64, "mixed": cs.CS_MIXED_BF16}[name]
        ctx = cs.cs_basis_init(w.R, w.lmax, w.nmax, w.n_r, w.n_theta, w.n_phi, 0, idx)
        if prec != cs.CS_FP64:  # double-float Rayleigh-Ritz apply and dense work
            cs.cs_set_rr_precision(ctx, cs.CS_DF64)
            cs.cs_set_dense_precision(ctx, cs.CS_DF64)
        xyz = torch.tensor(cs.grid_points(ctx), device=dev)
        v_ext = erf_cluster_potential_t(xyz, atoms, Z, w.extra["rc"]).contiguous()
        rho0 = gaussian_atom_density_t(xyz, atoms, Z, 1.0).contiguous()
        v0 = torch.tensor(W.gaussian(17, ctx.d), device=dev)
        p = cs.ScfParams(n_s=w.n_s, n_want=w.n_want, degree=w.degree, filter_prec=prec,
                         n_electrons=Z * len(atoms), kT=6.3e-4, beta=0.3, history=8,
                         first_tol=1e-3, first_max_iter=40, lanczos_k=10, e_ion=e_ion)
        S = cs.cs_scf_create(ctx, p, v_ext, rho0, v0)
        X = torch.tensor(W.gaussian_block(w.x_seed, w.d, w.n_s).T.copy(), device=dev)
        theta = torch.empty(w.n_s, dtype=torch.float64, device=dev)
        resid = torch.empty_like(theta)
        S.work()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = []
        for _ in range(max_iter):
            reps.append(cs.cs_scf_step(S, X, theta, resid))
            if len(reps) > 1 and abs(reps[-1]["dE"]) <= tol:
                break
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        last = reps[-1]
        out[name] = {"seconds": round(sec, 3), "iterations": len(reps),
                     "converged": len(reps) > 1 and abs(last["dE"]) <= tol,
                     "ms_per_iteration": round(1e3 * sec / len(reps), 2),
                     "first_chfsi_iterations": reps[0]["chfsi_iterations"],
                     "energy": last["energy"], "energy_per_atom": last["energy"] / len(atoms),
                     "last_dE": last["dE"], "mu": last["mu"], "max_resid": last["max_resid"],
                     "dE_history": [r["dE"] for r in reps]}
        S.close()
        ctx.close()
    for name in precisions:
        if name != "fp64" and "fp64" in out:
            out[f"{name}_energy_minus_fp64"] = out[name]["energy"] - out["fp64"]["energy"]
    return out


def first_solve_measure(dev, tol=1e-4, n_want=64):
    """The first eigensolve of an SCF on the 32-atom cluster (fixed potential, the seeded random
    block of 80 states): time and iterations until the 64 lowest residuals are <= tol, for
    LOBPCG with and without the Teter-Payne-Allan preconditioner (FP64) and for ChFSI with the
    FP64 and the FP32 filter (double-float Rayleigh-Ritz)."""
    import torch

    import paper_1404_3773_gb300 as cs
    from workloads.device import erf_cluster_potential_t
    w = W.erf_cluster_32()
    idx = torch.device(dev).index or 0
    ctx = cs.cs_basis_init(w.R, w.lmax, w.nmax, w.n_r, w.n_theta, w.n_phi, 0, idx)
    xyz = torch.tensor(cs.grid_points(ctx), device=dev)
    cs.cs_set_potential(ctx, erf_cluster_potential_t(xyz, w.atoms(), w.extra["Z"],
                                                     w.extra["rc"]).contiguous())
    X0 = torch.tensor(W.gaussian_block(w.x_seed, w.d, w.n_s).T.copy(), device=dev)
    v0 = torch.tensor(W.gaussian(17, ctx.d), device=dev)
    theta = torch.empty(w.n_s, dtype=torch.float64, device=dev)
    resid = torch.empty_like(theta)
    out = {"workload": f"erf32_l30_n48, fixed potential, 80 random states, stop when the "
                       f"{n_want} lowest residuals are <= {tol:g}"}
    for name, pre in (("lobpcg_tpa", True), ("lobpcg_none", False)):
        X = X0.clone()
        work = torch.empty(cs.cs_lobpcg_workspace_bytes(ctx, w.n_s), dtype=torch.uint8,
                           device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, rs = cs.cs_lobpcg(ctx, X, n_want, theta, resid, tol=tol, max_iter=150,
                              precondition=pre, work=work, raise_not_converged=False)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        out[name] = {"seconds": round(sec, 3), "iterations": it, "restarts": rs,
                     "max_resid": float(resid[:n_want].max())}
        del work
    for name, prec, rr in (("chfsi_fp64", cs.CS_FP64, cs.CS_FP64),
                           ("chfsi_fp32_rr_df64", cs.CS_FP32, cs.CS_DF64)):
        cs.cs_set_rr_precision(ctx, rr)
        cs.cs_set_dense_precision(ctx, rr)
        X = X0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it = cs.cs_chfsi(ctx, X, n_want, w.degree, v0, theta, resid, tol=tol, max_iter=60,
                         precision=prec, raise_not_converged=False)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        out[name] = {"seconds": round(sec, 3), "iterations": it,
                     "max_resid": float(resid[:n_want].max())}
    ctx.close()
    return out


def eigen_gate_measure(dev):
    """The mixed form's acceptance gate on the 32-atom cluster: ChFSI from the seeded block
    with the all-FP64 path to residuals of 1e-8, then with the bench's filter precisions
    (double-float Rayleigh-Ritz and Gram/rotations) for as many iterations as FP64 took plus
    ten; the largest deviation of the 64 lowest Ritz values from FP64 (gate: 1e-6 Ha)."""
    import torch

    import paper_1404_3773_gb300 as cs
    from workloads.device import erf_cluster_potential_t
    w = W.erf_cluster_32()
    idx = torch.device(dev).index or 0
    ctx = cs.cs_basis_init(w.R, w.lmax, w.nmax, w.n_r, w.n_theta, w.n_phi, 0, idx)
    xyz = torch.tensor(cs.grid_points(ctx), device=dev)
    cs.cs_set_potential(ctx, erf_cluster_potential_t(xyz, w.atoms(), w.extra["Z"],
                                                     w.extra["rc"]).contiguous())
    X0 = torch.tensor(W.gaussian_block(w.x_seed, w.d, w.n_s).T.copy(), device=dev)
    v0 = torch.tensor(W.gaussian(2003, ctx.d), device=dev)
    th64 = torch.empty(w.n_s, dtype=torch.float64, device=dev)
    r64 = torch.empty_like(th64)
    it64 = cs.cs_chfsi(ctx, X0.clone(), w.n_want, w.degree, v0, th64, r64, tol=1e-8,
                       max_iter=80, precision=cs.CS_FP64)
    out = {"workload": "erf32_l30_n48 ChFSI from the seeded block, 64 lowest Ritz values",
           "fp64_iterations": it64, "gate_ha": 1e-6}
    cs.cs_set_rr_precision(ctx, cs.CS_DF64)
    cs.cs_set_dense_precision(ctx, cs.CS_DF64)
    for name, prec in (("mixed", cs.CS_MIXED_BF16), ("fp32", cs.CS_FP32)):
        th = torch.empty_like(th64)
        rr = torch.empty_like(th64)
        it = cs.cs_chfsi(ctx, X0.clone(), w.n_want, w.degree, v0, th, rr, tol=1e-8,
                         max_iter=it64 + 10, precision=prec, raise_not_converged=False)
        dmax = float(np.max(np.abs(th.cpu().numpy()[:w.n_want] - th64.cpu().numpy()[:w.n_want])))
        out[name] = {"iterations": it, "max_dev_vs_fp64_ha": dmax,
                     "max_resid": float(rr[:w.n_want].max()), "within_gate": dmax < 1e-6}
    ctx.close()
    return out


def _bond_midpoints(atoms, rcut):
    """Midpoints of the atom pairs closer than rcut (bohr): centres of the bond functions."""
    mids = [(atoms[a] + atoms[b]) / 2.0 for a in range(len(atoms)) for b in range(a + 1, len(atoms))
            if np.linalg.norm(atoms[a] - atoms[b]) < rcut]
    return np.array(mids, dtype=np.float64).reshape(-1, 3)


def _center_features(cs, atoms, mids, mu, width):
    """Network inputs of every centre: the radial descriptor (the atom's neighbours; for a bond
    midpoint, every atom) and a flag that marks bond centres."""
    fa = cs.cs_atom_descriptors(atoms, mu, width)
    fb = [cs.cs_atom_descriptors(np.vstack([m[None, :], atoms]), mu, width)[0] for m in mids]
    F = np.zeros((len(atoms) + len(mids), len(mu) + 1))
    F[:len(atoms), :len(mu)] = fa
    if len(mids):
        F[len(atoms):, :len(mu)] = np.array(fb)
        F[len(atoms):, len(mu)] = 1.0
    return F


def learned_init_measure(dev, n_train=160, n_test=40, tol=1e-6, hidden=128, steps=3000,
                         ceiling=True, rcut=4.0, ridge=1e-4, n_val=24):
    """The learned initial density: small clusters of 4-12 Z=4 erf pseudo-atoms (R = 9, lmax 10,
    16 radial functions, 32 x 22 x 42 grid), SCF (mixed filter) from the Gaussian start to
    |dE| <= tol. The correction to the start is expanded in unit-integral Gaussians on every
    atom and on the midpoint of every pair closer than rcut (bond functions: the converged
    density gains bonding charge between atoms, which atom-centred spherical functions cannot
    hold). On the training clusters the converged density minus the start is fitted by these
    functions (weighted least squares); a 17-128-128-128-5 tanh network learns the fitted
    coefficients from each centre's radial descriptor and a bond flag (Adam). On the held-out
    clusters the SCF runs from the Gaussian start, from the learned start, and (ceiling) from
    the cluster's own best fit. The fits are ridge-regularised (ridge tr(M)/n |c|^2): the atom
    and bond Gaussians overlap, and unregularised fits cancel large coefficients that a network
    cannot learn. The learned start is the Gaussian start plus alpha times the predicted
    correction, clipped at zero and renormalised to the electron count. alpha is chosen on the
    last n_val training clusters, which the network does not see: the value of (0, 0.25, 0.5,
    0.75, 1) with the fewest SCF iterations there; alpha = 0 is the fallback to the Gaussian
    start. A cluster also falls back if the integral of |predicted correction| per electron
    exceeds twice the largest value among the training clusters' own fits (a prediction outside
    what training saw)."""
    import torch

    import paper_1404_3773_gb300 as cs
    from workloads.device import erf_cluster_potential_t, gaussian_atom_density_t
    idx = torch.device(dev).index or 0
    ctx = cs.cs_basis_init(9.0, 10, 16, 32, 22, 42, 0, idx)
    cs.cs_set_rr_precision(ctx, cs.CS_DF64)
    cs.cs_set_dense_precision(ctx, cs.CS_DF64)
    xyz = torch.tensor(cs.grid_points(ctx), device=dev)
    mu = np.linspace(2.0, 10.0, 16)
    width = 0.5
    sig = np.array([0.6, 0.9, 1.3, 1.9, 2.8])

    def cluster(i):
        natoms = 4 + int(9 * W.uniform(5000 + i, 1)[0])
        return W.place_atoms(5100 + i, natoms, 3.5, 2.2)

    def scf(atoms, rho0):
        ne = 4.0 * len(atoms)
        n_s = int(ne // 2) + 8
        v_ext = erf_cluster_potential_t(xyz, atoms, 4.0, 0.8).contiguous()
        p = cs.ScfParams(n_s=n_s, n_want=int(ne // 2), degree=12, filter_prec=cs.CS_MIXED_BF16,
                         n_electrons=ne, kT=6.3e-4, beta=0.3, history=8, first_tol=1e-3,
                         first_max_iter=40, lanczos_k=10, e_ion=0.0, first_solver=0)
        S = cs.cs_scf_create(ctx, p, v_ext, rho0.contiguous(),
                             torch.tensor(W.gaussian(17, ctx.d), device=dev))
        X = torch.tensor(W.gaussian_block(18, ctx.d, n_s).T.copy(), device=dev)
        th = torch.empty(n_s, dtype=torch.float64, device=dev)
        rs = torch.empty_like(th)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it = 0
        for it in range(1, 101):
            rep = cs.cs_scf_step(S, X, th, rs)
            if it > 1 and abs(rep["dE"]) <= tol:
                break
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        rho = cs.cs_scf_grid(S, 1)
        S.close()
        return it, sec, rho, rep["energy"]

    def centres(atoms):
        mids = _bond_midpoints(atoms, rcut)
        return np.vstack([atoms, mids]), mids

    # training data
    D, C = [], []
    n_bonds = 0
    corr_max = 0.0  # largest integral of |fitted correction| per electron in training
    for i in range(n_train):
        atoms = cluster(i)
        start = gaussian_atom_density_t(xyz, atoms, 4.0, 1.0).contiguous()
        _, _, rho, _ = scf(atoms, start)
        cen, mids = centres(atoms)
        n_bonds += len(mids)
        cfit = cs.cs_fit_atom_density(ctx, cen, sig, (rho - start).contiguous(), ridge=ridge)
        corr = torch.zeros_like(start)
        cs.cs_atom_density(ctx, cen, sig, cfit, corr)
        corr_max = max(corr_max, cs.cs_grid_integrals(ctx, [corr.abs().contiguous()])[0] /
                       (4.0 * len(atoms)))
        C.append(cfit)
        D.append(_center_features(cs, atoms, mids, mu, width))
    n_fit_centres = sum(len(centres(cluster(i))[0]) for i in range(n_train - n_val))
    D_all, C_all = np.concatenate(D), np.concatenate(C)
    D, C = D_all[:n_fit_centres], C_all[:n_fit_centres]
    d_mean, d_std = D.mean(axis=0), D.std(axis=0) + 1e-6
    c_scale = float(np.abs(C).max()) or 1.0
    dims = [D.shape[1], hidden, hidden, hidden, len(sig)]
    params = []
    for k in range(len(dims) - 1):
        params.append((W.gaussian_block(5200 + k, dims[k], dims[k + 1])
                       / math.sqrt(dims[k])).ravel(order="F"))
        params.append(np.zeros(dims[k + 1]))
    net = cs.cs_mlp_create(dims, np.concatenate(params).astype(np.float32), max_rows=D.shape[0],
                           cuda_device=idx)
    Xd = torch.tensor(((D - d_mean) / d_std).T.copy(), dtype=torch.float32, device=dev)
    Td = torch.tensor((C / c_scale).T.copy(), dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    loss0 = cs.cs_mlp_train_step(net, Xd, Td, 1e-3)
    for _ in range(steps):
        cs.cs_mlp_train_step(net, Xd, Td, 1e-3, want_loss=False)
    loss = cs.cs_mlp_loss_grad(net, Xd, Td)[0]
    train_s = time.perf_counter() - t0
    # the same loss on the validation clusters' centres (not trained on)
    Dv, Cv = D_all[n_fit_centres:], C_all[n_fit_centres:]
    val_loss = None
    if Dv.shape[0] > 0:
        Xv = torch.tensor(((Dv - d_mean) / d_std).T.copy(), dtype=torch.float32, device=dev)
        Tv = torch.tensor((Cv / c_scale).T.copy(), dtype=torch.float32, device=dev)
        val_loss = cs.cs_mlp_loss_grad(net, Xv, Tv)[0]
    def learned_start(atoms, start, alpha):
        """(density, accepted): start + alpha * prediction, clipped at 0, renormalised"""
        ne = 4.0 * len(atoms)
        cen, mids = centres(atoms)
        feats = (_center_features(cs, atoms, mids, mu, width) - d_mean) / d_std
        coef = cs.cs_mlp_forward(net, torch.tensor(feats.T.copy(), dtype=torch.float32,
                                                   device=dev)).cpu().numpy().T * c_scale
        corr = torch.zeros_like(start)
        cs.cs_atom_density(ctx, cen, sig, coef.astype(np.float64), corr)
        if cs.cs_grid_integrals(ctx, [corr.abs().contiguous()])[0] / ne > 2.0 * corr_max:
            return start, False
        rho = torch.clamp(start + alpha * corr, min=0.0).contiguous()
        rho *= ne / cs.cs_grid_integrals(ctx, [rho])[0]
        return rho, True

    # alpha on the validation clusters (not used to fit the network)
    alphas = (0.0, 0.25, 0.5, 0.75, 1.0)
    val_iters = {}
    for al in alphas:
        its = []
        for i in range(n_train - n_val, n_train):
            atoms = cluster(i)
            start = gaussian_atom_density_t(xyz, atoms, 4.0, 1.0).contiguous()
            rho0 = start if al == 0.0 else learned_start(atoms, start, al)[0]
            its.append(scf(atoms, rho0)[0])
        val_iters[al] = float(np.mean(its))
    alpha = min(alphas, key=lambda x: (val_iters[x], x))
    # held-out comparison
    it_g, it_l, s_g, s_l, de, it_c, fell_back = [], [], [], [], [], [], 0
    for i in range(n_train, n_train + n_test):
        atoms = cluster(i)
        ne = 4.0 * len(atoms)
        start = gaussian_atom_density_t(xyz, atoms, 4.0, 1.0).contiguous()
        a, sa, rho_c, ea = scf(atoms, start)
        cen, mids = centres(atoms)
        if ceiling:  # start from this cluster's own best-fit correction
            cfit = cs.cs_fit_atom_density(ctx, cen, sig, (rho_c - start).contiguous(), ridge=ridge)
            fitted = start.clone()
            cs.cs_atom_density(ctx, cen, sig, cfit, fitted)
            fitted *= ne / cs.cs_grid_integrals(ctx, [fitted])[0]
            it_c.append(scf(atoms, fitted)[0])
        learned, ok = learned_start(atoms, start, alpha) if alpha > 0.0 else (start, False)
        if ok:
            b, sb, _, eb = scf(atoms, learned)
        else:  # fallback: the Gaussian start
            fell_back += 1
            b, sb, eb = a, sa, ea
        it_g.append(a)
        it_l.append(b)
        s_g.append(sa)
        s_l.append(sb)
        de.append(abs(ea - eb) / len(atoms))
    net.close()
    ctx.close()
    return {"workload": f"{n_train - n_val} training + {n_val} validation + {n_test} held-out "
                        "clusters of 4-12 Z=4 erf atoms "
                        "(R 9, lmax 10, N 16, grid 32x22x42), mixed-filter SCF to "
                        f"|dE| <= {tol:g} Ha; correction on atoms and on bond midpoints "
                        f"(pairs closer than {rcut:g} bohr)",
            "train_centres": int(D.shape[0]), "train_bond_centres": int(n_bonds),
            "train_loss_first": loss0, "train_loss_final": loss, "validation_loss": val_loss,
            "train_seconds": round(train_s, 3),
            "held_out_mean_iterations_gaussian_start": float(np.mean(it_g)),
            "held_out_mean_iterations_learned_start": float(np.mean(it_l)),
            "held_out_mean_seconds_gaussian_start": round(float(np.mean(s_g)), 4),
            "held_out_mean_seconds_learned_start": round(float(np.mean(s_l)), 4),
            "held_out_max_energy_difference_per_atom_ha": float(np.max(de)),
            "held_out_fallbacks": fell_back,
            "validation_mean_iterations_by_alpha": {str(k): v for k, v in val_iters.items()},
            "alpha": alpha,
            "train_max_abs_correction_per_electron": corr_max,
            "held_out_mean_iterations_own_fit_start": float(np.mean(it_c)) if it_c else None}


def batched_measure(dev, reps=2):
    """96 clusters of 4-48 erf atoms (R 8-16, lmax 12-32, N 24-56, up to 128 states each),
    FP32 degree-16 filter: one persistent graph-captured launch per Chebyshev step for the
    whole batch (autotuned angular tiles) against 96 sequential single-cluster filters.
    Returns applies/s of both (state columns x degree / filter time)."""
    import torch

    import paper_1404_3773_gb300 as cs
    ws = W.batched_clusters(96)
    gen = torch.Generator(device=dev)
    gen.manual_seed(4000)
    ctxs, Xs, bounds = [], [], []
    for w in ws:
        ctx = cs.cs_basis_init(w.R, w.lmax, w.nmax, w.n_r, w.n_theta, w.n_phi, 0,
                               torch.device(dev).index or 0)
        xyz = torch.tensor(cs.grid_points(ctx), device=dev)
        v = torch.zeros(xyz.shape[0], dtype=torch.float64, device=dev)
        for a in torch.tensor(w.atoms(), device=dev):
            r = torch.linalg.norm(xyz - a, dim=1)
            x = r / 0.8
            v += torch.where(x < 1e-3, -4.0 * 2.0 / (0.8 * math.sqrt(math.pi)) * (1 - x * x / 3),
                             -4.0 * torch.special.erf(x) / torch.clamp(r, min=1e-300))
        cs.cs_set_potential(ctx, v.contiguous())
        X = torch.randn((w.n_s, ctx.d), generator=gen, device=dev, dtype=torch.float32)
        v0 = torch.randn(ctx.d, generator=gen, device=dev, dtype=torch.float64)
        b, tmin = cs.cs_lanczos_bound(ctx, v0, 10)
        bounds.append((tmin + (b - tmin) / 10.0, b, tmin))
        ctxs.append(ctx)
        Xs.append(X)
    degree = ws[0].degree
    a, b, a0 = (list(t) for t in zip(*bounds))
    batch = cs.cs_batch_create(ctxs, [w.n_s for w in ws], degree)
    variant, tune_ms = cs.cs_batch_tune(batch, Xs, a, b, a0)
    variant_ms = cs.cs_batch_tune_times(batch)
    nbytes = max(cs.cs_workspace_bytes(c, w.n_s, cs.CS_FP32) for c, w in zip(ctxs, ws))
    work_seq = torch.empty(nbytes, dtype=torch.uint8, device=dev)  # shared, calls are serial
    stream = torch.cuda.current_stream()
    cols = sum(w.n_s for w in ws) * degree
    Y = [X.clone() for X in Xs]
    cs.cs_batch_cheb_filter(batch, Y, a, b, a0)  # warm
    torch.cuda.synchronize()
    n0 = cs.cs_launch_count(ctxs[0])
    cs.cs_batch_cheb_filter(batch, Y, a, b, a0)
    torch.cuda.synchronize()
    launches_per_filter = cs.cs_launch_count(ctxs[0]) - n0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        cs.cs_batch_cheb_filter(batch, Y, a, b, a0)
    e1.record(stream)
    e1.synchronize()
    t_batch = e0.elapsed_time(e1) / reps
    Y2 = [X.clone() for X in Xs]
    for c, y, w, aa, bb, aa0 in zip(ctxs, Y2, ws, a, b, a0):  # warm
        cs.cs_cheb_filter(c, y, degree, aa, bb, aa0, cs.CS_FP32, work_seq)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        for c, y, w, aa, bb, aa0 in zip(ctxs, Y2, ws, a, b, a0):
            cs.cs_cheb_filter(c, y, degree, aa, bb, aa0, cs.CS_FP32, work_seq)
    e1.record(stream)
    e1.synchronize()
    t_seq = e0.elapsed_time(e1) / reps
    # same arithmetic in both forms: the filtered blocks agree
    Y3 = [X.clone() for X in Xs]
    cs.cs_batch_cheb_filter(batch, Y3, a, b, a0)
    Y4 = [X.clone() for X in Xs]
    for c, y, w, aa, bb, aa0 in zip(ctxs, Y4, ws, a, b, a0):
        cs.cs_cheb_filter(c, y, degree, aa, bb, aa0, cs.CS_FP32, work_seq)
    torch.cuda.synchronize()
    same = all(torch.equal(p, q) for p, q in zip(Y3, Y4))
    # the mixed precision (split-BF16 tensor-core kernels): concurrent batch against 96
    # sequential mixed filters
    nbytes_m = max(cs.cs_workspace_bytes(c, w.n_s, cs.CS_MIXED_BF16) for c, w in zip(ctxs, ws))
    work_m = torch.empty(nbytes_m, dtype=torch.uint8, device=dev)
    cs.cs_batch_set_precision(batch, cs.CS_MIXED_BF16)
    Ym = [X.clone() for X in Xs]
    cs.cs_batch_cheb_filter(batch, Ym, a, b, a0)  # capture + warm
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        cs.cs_batch_cheb_filter(batch, Ym, a, b, a0)
    e1.record(stream)
    e1.synchronize()
    t_bm = e0.elapsed_time(e1) / reps
    Ys = [X.clone() for X in Xs]
    for c, y, w, aa, bb, aa0 in zip(ctxs, Ys, ws, a, b, a0):  # warm
        cs.cs_cheb_filter(c, y, degree, aa, bb, aa0, cs.CS_MIXED_BF16, work_m)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        for c, y, w, aa, bb, aa0 in zip(ctxs, Ys, ws, a, b, a0):
            cs.cs_cheb_filter(c, y, degree, aa, bb, aa0, cs.CS_MIXED_BF16, work_m)
    e1.record(stream)
    e1.synchronize()
    t_sm = e0.elapsed_time(e1) / reps
    Y5 = [X.clone() for X in Xs]
    cs.cs_batch_cheb_filter(batch, Y5, a, b, a0)
    Y6 = [X.clone() for X in Xs]
    for c, y, w, aa, bb, aa0 in zip(ctxs, Y6, ws, a, b, a0):
        cs.cs_cheb_filter(c, y, degree, aa, bb, aa0, cs.CS_MIXED_BF16, work_m)
    torch.cuda.synchronize()
    same_m = all(torch.equal(p, q) for p, q in zip(Y5, Y6))
    # where the sequential time goes: each cluster's mixed filter alone (CUDA events), sorted.
    # Overlapping clusters can hide only the time of those that leave the GPU idle; the largest
    # ones fill it alone, so their share bounds what batching can gain.
    per = []
    for c, y, w, aa, bb, aa0 in zip(ctxs, Ys, ws, a, b, a0):
        e0.record(stream)
        cs.cs_cheb_filter(c, y, degree, aa, bb, aa0, cs.CS_MIXED_BF16, work_m)
        e1.record(stream)
        e1.synchronize()
        per.append((e0.elapsed_time(e1), w.n_s, w.lmax))
    per.sort(reverse=True)
    tot = sum(p[0] for p in per)
    shares = {f"largest_{k}": round(sum(p[0] for p in per[:k]) / tot, 3) for k in (8, 16, 32)}
    mixed_clusters = {"sequential_ms_sum": round(tot, 3), "time_share": shares,
                      "largest_ms": [round(p[0], 3) for p in per[:8]],
                      "largest_n_s_lmax": [[p[1], p[2]] for p in per[:8]],
                      "median_ms": round(per[len(per) // 2][0], 3)}
    mixed = {"applies_per_s": round(cols / (t_bm / 1e3), 1),
             "sequential_applies_per_s": round(cols / (t_sm / 1e3), 1),
             "speedup_vs_sequential": round(t_sm / t_bm, 3),
             "filter_ms": round(t_bm, 3), "sequential_filter_ms": round(t_sm, 3),
             "variant": "concurrent", "bitwise_equal_to_sequential": bool(same_m),
             "clusters": mixed_clusters}
    return {"workload": "96 erf clusters (4-48 atoms, R 8-16, lmax 12-32, N 24-56, "
                        f"{sum(w.n_s for w in ws)} states in total), FP32 degree-{degree} filter",
            "applies_per_s": round(cols / (t_batch / 1e3), 1),
            "sequential_applies_per_s": round(cols / (t_seq / 1e3), 1),
            "speedup_vs_sequential": round(t_seq / t_batch, 3),
            "filter_ms": round(t_batch, 3), "sequential_filter_ms": round(t_seq, 3),
            "tuned_variant": cs.BATCH_VARIANTS[variant],
            "tune_filter_ms": {k: round(v, 3) for k, v in variant_ms.items()},
            "bitwise_equal_to_sequential": bool(same),
            "launches_per_filter": launches_per_filter,
            "mixed": mixed}


def at_scale_measure(dev, chunk=128):
    """The 400-atom cluster with Kleinman-Bylander s and p projectors (R = 26, lmax 60, 96 radial
    functions, d = 357216, 192 x 120 x 240 grid, 1600 projectors): one H.X on a chunk of 128
    states in each precision (CUDA events, after a warm-up call), the split-BF16 and FP32
    errors against the FP64 product, and the per-class device times of the mixed call."""
    import torch

    import paper_1404_3773_gb300 as cs
    from workloads.device import erf_cluster_potential_t, kb_couplings, kb_projector_values_t
    w = W.erf_cluster_400_kb()
    idx = torch.device(dev).index or 0
    t_setup = time.time()
    ctx = cs.cs_basis_init(w.R, w.lmax, w.nmax, w.n_r, w.n_theta, w.n_phi, 0, idx)
    xyz = torch.tensor(cs.grid_points(ctx), device=dev)
    atoms = w.atoms()
    cs.cs_set_potential(ctx, erf_cluster_potential_t(xyz, atoms).contiguous())
    pcoef = torch.empty((4 * len(atoms), ctx.d), dtype=torch.float64, device=dev)
    per = 16
    for a0 in range(0, len(atoms), per):
        cnt = min(per, len(atoms) - a0)
        pg = kb_projector_values_t(xyz, atoms, rc=1.0, first=a0, count=cnt)
        pg = pg.reshape(4 * cnt, ctx.n_r, ctx.n_theta, ctx.n_phi).contiguous()
        cs.cs_forward_transform(ctx, pg, pcoef[4 * a0:4 * (a0 + cnt)])
        del pg
    cs.cs_set_projectors(ctx, pcoef, kb_couplings(len(atoms)))
    del pcoef, xyz
    torch.cuda.synchronize()
    t_setup = time.time() - t_setup
    X = torch.tensor(np.ascontiguousarray(W.gaussian_block(w.x_seed, ctx.d, chunk).T), device=dev)
    out = {}
    prods = {}
    stream = torch.cuda.current_stream()
    for name, prec in (("mixed", cs.CS_MIXED_BF16), ("fp32", cs.CS_FP32), ("fp64", cs.CS_FP64)):
        Xp = X if prec == cs.CS_FP64 else X.float()
        Y = torch.empty_like(Xp)
        work = ctx.workspace(chunk, prec)
        cs.cs_apply_H(ctx, Xp, Y, prec, work)  # warm
        torch.cuda.synchronize()
        if name == "mixed":
            cs.cs_profile_begin(ctx)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cs.cs_apply_H(ctx, Xp, Y, prec, work)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        entry = {"ms_per_apply_block": round(ms, 3), "applies_per_s": round(chunk / (ms / 1e3), 1)}
        if name == "mixed":
            pms, pn = cs.cs_profile_end(ctx)
            names = cs.profile_class_names()
            entry["class_ms"] = {names[i]: round(pms[i], 3) for i in range(len(names)) if pn[i]}
        out[name] = entry
        prods[name] = Y.double()
        del work
        ctx._ws.clear()
        torch.cuda.empty_cache()
    ref = prods["fp64"]
    for name in ("mixed", "fp32"):
        out[name]["rel_error_vs_fp64"] = float(torch.linalg.norm(prods[name] - ref) /
                                               torch.linalg.norm(ref))
    out["workload"] = ("erf400kb_l60_n96: 400 erf atoms + s,p projectors (1600), R=26, lmax=60, "
                       f"96 radial fns/l, d={ctx.d}, grid 192x120x240, {chunk}-state chunk")
    out["setup_s"] = round(t_setup, 1)
    ctx.close()
    return out


def at_scale_chfsi_measure(dev, chunk=128, timed_iters=2, cpu_seconds=10.0):
    """ChFSI iterations on the 400-atom cluster with s and p projectors (R = 26, lmax 60, 96
    radial functions, d = 357216, 192 x 120 x 240 grid, 1600 projectors), 880 states, degree
    20: the mixed filter in residual form over chunks of 128 states (19 split-BF16 H.X per
    state), then Cholesky-QR twice and Rayleigh-Ritz over all 880 states with a double-float
    H.X (FP64-class; its projector pair as exact slice products) and the Gram matrices and
    rotations as exact slice products on the tensor cores (FP64 factorisation, eigensolve and
    residuals).
    The block starts random (seeded); one untimed iteration with the first-pass interval
    (Lanczos bounds), then `timed_iters` timed iterations (CUDA events, per-class device
    times). Every call goes through the C ABI."""
    import torch

    import paper_1404_3773_gb300 as cs
    from workloads.device import erf_cluster_potential_t, kb_couplings, kb_projector_values_t
    w = W.erf_cluster_400_kb()
    n_s, degree = w.n_s, w.degree
    idx = torch.device(dev).index or 0
    t_setup = time.time()
    ctx = cs.cs_basis_init(w.R, w.lmax, w.nmax, w.n_r, w.n_theta, w.n_phi, 0, idx)
    xyz = torch.tensor(cs.grid_points(ctx), device=dev)
    atoms = w.atoms()
    cs.cs_set_potential(ctx, erf_cluster_potential_t(xyz, atoms).contiguous())
    pcoef = torch.empty((4 * len(atoms), ctx.d), dtype=torch.float64, device=dev)
    per = 16
    for f in range(0, len(atoms), per):
        cnt = min(per, len(atoms) - f)
        pg = kb_projector_values_t(xyz, atoms, rc=1.0, first=f, count=cnt)
        pg = pg.reshape(4 * cnt, ctx.n_r, ctx.n_theta, ctx.n_phi).contiguous()
        cs.cs_forward_transform(ctx, pg, pcoef[4 * f:4 * (f + cnt)])
        del pg
    cs.cs_set_projectors(ctx, pcoef, kb_couplings(len(atoms)))
    del pcoef, xyz
    ctx._ws.clear()
    torch.cuda.empty_cache()
    cs.cs_set_rr_precision(ctx, cs.CS_DF64)
    cs.cs_set_dense_precision(ctx, cs.CS_FP64_SLICED)
    gen = torch.Generator(device=dev)
    gen.manual_seed(w.x_seed)
    X = torch.randn((n_s, ctx.d), generator=gen, dtype=torch.float64, device=dev)
    v0 = torch.randn(ctx.d, generator=gen, dtype=torch.float64, device=dev)
    HX = torch.empty_like(X)
    theta = torch.empty(n_s, dtype=torch.float64, device=dev)
    resid = torch.empty_like(theta)
    work = ctx.workspace(n_s, cs.CS_MIXED_BF16)
    torch.cuda.synchronize()
    t_setup = time.time() - t_setup
    b, tmin = cs.cs_lanczos_bound(ctx, v0, 10, work)
    stream = torch.cuda.current_stream()

    def iteration(a, a0):
        for c0 in range(0, n_s, chunk):
            c1 = min(n_s, c0 + chunk)
            cs.cs_cheb_filter_ritz(ctx, X[c0:c1], HX[c0:c1], theta[c0:c1], degree, a, b, a0,
                                   cs.CS_MIXED_BF16, work)
        cs.cs_cholqr(ctx, X, work)
        cs.cs_rayleigh_ritz(ctx, X, theta, resid, HX, work)

    # the random block: Cholesky-QR and Rayleigh-Ritz give its Ritz values and H X, then the
    # first iteration with the first-pass interval
    t0 = time.time()
    cs.cs_cholqr(ctx, X, work)
    cs.cs_rayleigh_ritz(ctx, X, theta, resid, HX, work)
    iteration(tmin + (b - tmin) / 10.0, tmin)
    torch.cuda.synchronize()
    first_s = time.time() - t0
    hist = [float(resid[:w.n_want].max())]
    times = []
    cs.cs_profile_begin(ctx)
    for _ in range(timed_iters):
        th = theta.cpu().numpy()
        a, a0 = float(th[-1]), float(th[0])
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        iteration(a, a0)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        hist.append(float(resid[:w.n_want].max()))
    pms, pn = cs.cs_profile_end(ctx)
    names = cs.profile_class_names()
    ms = sum(times) / len(times)
    hx_per_iter = degree  # degree - 1 filter products + the Rayleigh-Ritz one, per state
    applies = hx_per_iter * n_s
    # ---- end to end through the public API: the block, its H X and Ritz values in from pinned
    # host memory, the same out
    Xh, HXh, thh = X.cpu().pin_memory(), HX.cpu().pin_memory(), theta.cpu().pin_memory()
    th_np = thh.numpy().copy()
    a, a0 = float(th_np[-1]), float(th_np[0])
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    X.copy_(Xh, non_blocking=True)
    HX.copy_(HXh, non_blocking=True)
    theta.copy_(thh, non_blocking=True)
    iteration(a, a0)
    Xh.copy_(X, non_blocking=True)
    HXh.copy_(HX, non_blocking=True)
    thh.copy_(theta, non_blocking=True)
    e1.record(stream)
    e1.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    hist.append(float(resid[:w.n_want].max()))
    # per-class device time over the timed iterations, and the dominant single-kernel class
    # rated against its pipe (the lmax-60 angular block runs on the FP32 pipe)
    classes = {}
    for i, nm in enumerate(names):
        if pn[i]:
            classes[nm] = {"ms_per_iteration": round(pms[i] / timed_iters, 3),
                           "launches_per_iteration": pn[i] / timed_iters,
                           "share": round(pms[i] / max(1e-9, sum(pms)), 4)}
    L, N, nr, nt, nph = w.L, w.nmax, w.n_r, w.n_theta, w.n_phi
    f_leg = 2.0 * nt * L * L * nr / 2.0
    f_phi = 2.5 * nph * math.log2(nph) * nr * nt
    ang_flops_state = 2 * f_leg + 2 * f_phi + float(nr * nt * nph)
    roof = None
    single = {k: v for k, v in classes.items() if not k.startswith("dense")}
    if single:
        dom = max(single, key=lambda k: single[k]["ms_per_iteration"])
        n_launch = pn[names.index(dom)]
        avg_ms = pms[names.index(dom)] / n_launch
        if dom == "angular_df64":
            # the Rayleigh-Ritz H.X: one launch over all states, double-float on the FP32 pipe
            per_launch = ang_flops_state * n_s / max(1.0, pn[names.index(dom)] / timed_iters)
            ach = per_launch / (avg_ms / 1e3) / 1e12
            roof = {"bound": "alu", "kernel": dom, "achieved": round(ach, 4),
                    "peak": round(DF64_PEAK_TFLOPS, 3), "unit": "TFLOP/s",
                    "frac": round(ach / DF64_PEAK_TFLOPS, 4), "traffic": None,
                    "flops_per_launch": per_launch, "avg_launch_ms": round(avg_ms, 4),
                    "peak_source": "FP32 issue rate / 15 instructions per double-float "
                                   "multiply-add"}
        elif dom == "angular_f32":
            # the mixed filter's angular block, one profiled record per H.X: at lmax 60 the
            # three-pass tensor-core block (Legendre sums, phi passes, Legendre quadrature)
            # unless CS_ANGULAR_KERNEL selects another
            env = os.environ.get("CS_ANGULAR_KERNEL", "")
            wide = env == "" or env.startswith("w")
            flops = ang_flops_state * chunk
            ach = flops / (avg_ms / 1e3) / 1e12
            peaks = measured_peaks()
            byts = 2.0 * w.n_r * L * L * chunk * 4  # G in, G' out (FP32)
            if wide:
                peak = peaks["bf16_tflops_sustained"] / 3.0
                src = (f"{peak_word(peaks)} bf16 sustained / 3 (split BF16: three BF16 products "
                       "per product)")
            else:
                peak, src = FP32_PEAK_TFLOPS, "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"
            roof = {"bound": "tensor" if wide else "alu", "kernel": dom,
                    "launches_per_hx": 3 if wide else 1, "achieved": round(ach, 4),
                    "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(ach / peak, 4),
                    "traffic": None, "flops_per_hx": flops, "ms_per_hx": round(avg_ms, 4),
                    "peak_source": src,
                    "hbm_view": {"algorithmic_bytes": byts,
                                 "achieved_gbs": round(byts / (avg_ms / 1e3) / 1e9, 1)},
                    "note": "flops per H.X include the last, ragged chunk's 112 states as 128"}
        else:
            roof = {"kernel": dom, "avg_launch_ms": round(avg_ms, 4), "frac": None}
    cpu = cpu_baseline_local(w, dev, budget_s=cpu_seconds)
    out = {"workload": f"erf400kb_l60_n96: 400 erf atoms + s,p projectors (1600), R=26, "
                       f"lmax=60, 96 radial fns/l, d={ctx.d}, grid 192x120x240, {n_s} states "
                       f"(filter in chunks of {chunk}), degree {degree}",
           "step": "one ChFSI iteration: residual-form mixed filter (19 split-BF16 H.X per "
                   "state) + CholQR x2 + Rayleigh-Ritz (double-float H.X with the projector pair "
                   "as slice products; Gram matrices and rotations as exact slice products on "
                   "the tensor cores; FP64 factorisation, eigensolve and residuals)",
           "ms_per_iteration": round(ms, 1),
           "iteration_ms": [round(t, 1) for t in times],
           "value": round(applies / (ms / 1e3), 1), "unit": "applies/s",
           "hx_per_iteration_per_state": hx_per_iter,
           "e2e": {"value": round(applies / (e2e_ms / 1e3), 1), "unit": "applies/s",
                   "h2d_bytes_per_step": 2 * X.numel() * 8 + n_s * 8,
                   "d2h_bytes_per_step": 2 * X.numel() * 8 + n_s * 8},
           "kernel_classes": classes, "roofline": roof, "cpu_baseline": cpu,
           "first_iteration_s": round(first_s, 2), "setup_s": round(t_setup, 1),
           "max_resid_800_lowest_by_iteration": hist}
    ctx.close()
    return out


def cpu_baseline_local(w, dev=None, budget_s=10.0, cols=1):
    """The FP64 oracle's H.X on `cols` state(s) of a workload's basis and grid with its local
    potential only, on the host cores, for about budget_s seconds. The projector pair is left
    out: the oracle would form its coefficients from grid values of every projector (1600 x
    5.5 million doubles for the 400-atom cluster, 70 GB). The seeded input generator
    evaluates the potential on the oracle's own grid points (with torch on `dev` when given:
    numpy takes over a minute for 400 atoms on 5.5 million points)."""
    from oracle.basis import basis_for
    from oracle.hamiltonian import Hamiltonian
    t0 = time.perf_counter()
    b = basis_for(w)
    pts = b.points()
    if dev is not None:
        import torch
        from workloads.device import erf_cluster_potential_t
        v = erf_cluster_potential_t(torch.tensor(pts, device=dev), w.atoms(),
                                    w.extra["Z"], w.extra["rc"]).cpu().numpy()
    else:
        v = w.potential_at(pts)
    H = Hamiltonian(b, v)
    setup = time.perf_counter() - t0
    X = w.x_block(cols)
    t0 = time.perf_counter()
    n = 0
    while True:
        H.apply(X)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": round(n * cols / el, 5), "unit": "applies/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{n} oracle H.X calls on {cols} state(s) of the same basis and grid, local "
                      f"potential only (no projectors); {el:.1f} s after {setup:.0f} s of set-up"}


def cpu_baseline(w, budget_s=15.0, cols=8):
    """The FP64 oracle as it stands, on the host cores: H.X on `cols` states of the same
    workload, repeated for about `budget_s` seconds. Returns applies/s (state columns per
    second)."""
    from oracle.basis import basis_for
    from oracle.hamiltonian import Hamiltonian
    b = basis_for(w)
    H = Hamiltonian(b, w.potential_at(b.points()))
    X = w.x_block(cols)
    H.apply(X)  # warm
    t0 = time.perf_counter()
    n = 0
    while True:
        H.apply(X)
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": round(n * cols / el, 4), "unit": "applies/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{n} oracle H.X calls on {cols} of the 80 states of the same workload "
                      f"(FP64, numpy; {el:.1f} s)"}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank, world, _ = _rank_env()
    if rank != 0:
        return
    w = W.erf_cluster_32()
    from oracle.basis import basis_for
    from oracle.hamiltonian import Hamiltonian
    b = basis_for(w)
    H = Hamiltonian(b, w.potential_at(b.points()))
    cols = 4
    X = w.x_block(cols)
    for _ in range(args.warmup):
        H.apply(X)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        H.apply(X)
    el = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    value = args.steps * cols / el
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4),
            "unit": "applies/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * el / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded erf pseudo-atom cluster and Gaussian state block)",
            "config": {"workload": "erf32_l30_n48 (same as the GPU arm)",
                       "step": f"one oracle H.X on {cols} of the 80 states (bounded sample)"},
            "cpu_baseline": {"value": round(value, 4), "unit": "applies/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{args.steps} oracle H.X calls on {cols} states"},
            "e2e": {"value": round(value, 4), "unit": "applies/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_hx(case, n_states, reps, precision="mixed"):
    """A small case for profiler captures (no JSON bench line): `reps` H.X calls (mixed, or
    double-float on FP64 states) on `n_states` seeded states of the 32-atom cluster (erf32) or
    of the 400-atom cluster without its projectors (erf400), after one untimed call; prints the
    mean CUDA-event time."""
    import torch

    import paper_1404_3773_gb300 as cs
    from workloads.device import erf_cluster_potential_t
    w = W.erf_cluster_32() if case == "erf32" else W.erf_cluster_400_kb()
    ctx = cs.cs_basis_init(w.R, w.lmax, w.nmax, w.n_r, w.n_theta, w.n_phi, 0, 0)
    xyz = torch.tensor(cs.grid_points(ctx), device="cuda")
    cs.cs_set_potential(ctx, erf_cluster_potential_t(xyz, w.atoms()).contiguous())
    del xyz
    gen = torch.Generator(device="cuda")
    gen.manual_seed(w.x_seed)
    prec = cs.CS_DF64 if precision == "df64" else cs.CS_MIXED_BF16
    dtype = torch.float64 if precision == "df64" else torch.float32
    X = torch.randn((n_states, ctx.d), generator=gen, dtype=dtype, device="cuda")
    Y = torch.empty_like(X)
    work = ctx.workspace(n_states, prec)
    cs.cs_apply_H(ctx, X, Y, prec, work)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        cs.cs_apply_H(ctx, X, Y, prec, work)
    e1.record()
    e1.synchronize()
    if cs.cs_device_error(ctx) != 0:
        raise RuntimeError("device error word set")
    print(json.dumps({"profile_hx": case, "precision": precision, "states": n_states, "reps": reps,
                      "ms_per_apply": round(e0.elapsed_time(e1) / max(1, reps), 4),
                      "angular_kernel": os.environ.get("CS_ANGULAR_KERNEL", "default")}))
    ctx.close()


def profile_dense(n_states, case="erf400"):
    """A case for profiler captures of the dense steps (no JSON bench line): one Cholesky-QR
    (two passes) and one Rayleigh-Ritz of `n_states` seeded FP64 states of the 400-atom
    cluster's basis (erf400, d = 357216; no projectors) or of the 32-atom cluster's (erf32,
    d = 46128: a few GB on the device, for full-section captures), with the dense precision of
    the at-scale iteration (slice products) and its double-float H.X; prints the CUDA-event
    times."""
    import torch

    import paper_1404_3773_gb300 as cs
    from workloads.device import erf_cluster_potential_t
    w = W.erf_cluster_32() if case == "erf32" else W.erf_cluster_400_kb()
    ctx = cs.cs_basis_init(w.R, w.lmax, w.nmax, w.n_r, w.n_theta, w.n_phi, 0, 0)
    xyz = torch.tensor(cs.grid_points(ctx), device="cuda")
    cs.cs_set_potential(ctx, erf_cluster_potential_t(xyz, w.atoms()).contiguous())
    del xyz
    cs.cs_set_rr_precision(ctx, cs.CS_DF64)
    cs.cs_set_dense_precision(ctx, cs.CS_FP64_SLICED)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(w.x_seed)
    X = torch.randn((n_states, ctx.d), generator=gen, dtype=torch.float64, device="cuda")
    HX = torch.empty_like(X)
    th = torch.empty(n_states, dtype=torch.float64, device="cuda")
    rs = torch.empty_like(th)
    work = ctx.workspace(n_states, cs.CS_MIXED_BF16)

    def timed(f):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        f()
        e1.record()
        e1.synchronize()
        return round(e0.elapsed_time(e1), 2)

    out = {"profile_dense": case, "states": n_states,
           "cholqr_ms": timed(lambda: cs.cs_cholqr(ctx, X, work))}
    cs.cs_profile_begin(ctx)
    out["rayleigh_ritz_ms"] = timed(lambda: cs.cs_rayleigh_ritz(ctx, X, th, rs, HX, work))
    pms, pn = cs.cs_profile_end(ctx)
    names = cs.profile_class_names()
    out["rayleigh_ritz_classes_ms"] = {nm: round(pms[i], 2) for i, nm in enumerate(names)
                                       if pn[i]}
    if cs.cs_device_error(ctx) != 0:
        raise RuntimeError("device error word set")
    print(json.dumps(out))
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "fp32", "mixed", "df64"],
                    help="filter precision")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--rr-precision", default="df64", choices=["same", "fp64", "df64"],
                    help="precision of the H X that Rayleigh-Ritz projects")
    ap.add_argument("--dense-precision", default="df64", choices=["fp64", "df64", "sliced"],
                    help="arithmetic of the Gram matrices and block rotations (sliced: exact "
                         "integer-slice products on the tensor cores, rounded once)")
    ap.add_argument("--form", default="ritz", choices=["ritz", "plain"],
                    help="filter form of the timed step: residual form from Ritz vectors "
                         "(steady state of a ChFSI loop) or the plain recurrence")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-at-scale", action="store_true")
    ap.add_argument("--no-at-scale-chfsi", action="store_true",
                    help="skip the ChFSI iterations of the 400-atom cluster (880 states)")
    ap.add_argument("--no-scf", action="store_true")
    ap.add_argument("--profile-hx", default=None, choices=["erf32", "erf400"],
                    help="only run a small mixed H.X case for profiler captures")
    ap.add_argument("--profile-states", type=int, default=32)
    ap.add_argument("--profile-reps", type=int, default=2)
    ap.add_argument("--profile-precision", default="mixed", choices=["mixed", "df64"],
                    help="arithmetic of the --profile-hx calls")
    ap.add_argument("--profile-dense", type=int, default=0, metavar="N",
                    help="only run one Cholesky-QR and one Rayleigh-Ritz of N states of the "
                         "400-atom cluster's basis for profiler captures")
    ap.add_argument("--profile-basis", default="erf400", choices=["erf32", "erf400"],
                    help="basis of --profile-dense")
    args = ap.parse_args()
    if args.profile_hx:
        profile_hx(args.profile_hx, args.profile_states, args.profile_reps,
                   args.profile_precision)
        return
    if args.profile_dense:
        profile_dense(args.profile_dense, args.profile_basis)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
