"""Benchmark: collision-operator evaluations per second on one GB300.

A step is one evaluation of Q(f) (the whole hot path: forward transform,
phase-weighted spectra and inverse transforms of every shifted field, cubic
products, accumulation over all M quadrature nodes) on the 3D N=64, M=2048
workload (32 radial x 8 x 8 cube directions, ring f = exp(-(|k|-3)^2), L=8).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is FP32 evaluations/s with f resident on the
device; `e2e` is the same through the host-buffer C-ABI call with the copies
inside the timed region.  L2 is flushed (256 MiB write) before every timed
step; per-step times come from CUDA events on the launching stream.  The
reference arm times the CPU FP64 oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import wke_inputs as I  # noqa: E402

METRIC = "Q(f) evals/s at 3D N=64 (FP32/split vs FP64 GPU, ≤1e-6 rel); serving p50/p99 ms"
UNIT = "evals/s"
WORKLOAD = I.WORKLOADS["3d_n64_m2048"]


def _config(precision="fp32"):
    w = WORKLOAD
    return {"workload": f"{w.name}: 3D N={w.N}, L={w.L}, M={w.M} ({w.n_r} radial x {w.n_s} x {w.n_sig} "
                        f"{w.sphere} directions), ring f=exp(-(|k|-3)^2), Nyquist kept",
            "d": w.d, "N": w.N, "M": w.M, "precision": precision,
            "l2": "flushed before every timed step (256 MiB write, outside the step events)"}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s in sm if mx and s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle

def _oracle_quad_args():
    from oracle import wke_oracle as O
    w = WORKLOAD
    return (w.d, w.n_r, w.n_s, w.n_sig, O.default_R(w.L), w.sphere)


def cpu_oracle_rate(pool, evals):
    """Evaluations/s of the FP64 oracle's fast form on the host cores: `evals`
    whole evaluations of the workload, each split over node ranges across the
    spawn pool's processes (oracle.pool) and summed in node order."""
    w = WORKLOAD
    f = w.initial()
    walls = []
    for _ in range(evals):
        _, wall, _ = pool.collision_fast(f, w.L, _oracle_quad_args())
        walls.append(wall)
    return evals / sum(walls), walls


def replica_rate(t_step_ms, world, device=None):
    """Whole-job rate of `world` independent replicas (one per GPU, each
    evaluating its own copy of the workload): the slowest rank's mean step
    time, taken with a MAX all-reduce, and world * 1000 / t_max evals/s."""
    t_max = t_step_ms
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([t_step_ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    return t_max, world * 1000.0 / t_max


def make_pool():
    from oracle.pool import OraclePool
    pool = OraclePool()
    return pool, pool.workers


# ------------------------------------------------------------------ GPU arm

def run_gpu(args, rank, world, pool, workers):
    import numpy as np
    import torch
    from paper_2503_12805_gb300 import wke

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = WORKLOAD
    f64 = w.initial()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def make(prec):
        return wke.Plan(w.d, w.N, w.L, w.n_r, w.n_s, w.n_sig, sphere=w.sphere, precision=prec,
                        chunk_bytes=int(args.chunk_mb * (1 << 20)))

    def timed(plan, f, Q, steps, warmup, profile=False):
        for _ in range(warmup):
            plan.collision(f, Q)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        if profile:
            wke.wke_plan_profile(plan.handle, True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        t0 = time.perf_counter()
        for i in range(steps):
            flush.fill_(i & 0xFF)                    # evict L2 between steps
            ev[i][0].record(stream)
            plan.collision(f, Q)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ms = [a.elapsed_time(b) for a, b in ev]
        prof = None
        if profile:
            prof = wke.wke_plan_profile_read(plan.handle)
            wke.wke_plan_profile(plan.handle, False)
        if world > 1:
            torch.distributed.barrier()
        return ms, wall, prof

    # measured FP32 and FP64 FMA rates of this GPU (the ALU roofs)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    with ClockSampler(dev.index) as pclk:
        peaks32 = wke.wke_alu_peak(wke.WKE_FP32, 5)
        peaks64 = wke.wke_alu_peak(wke.WKE_FP64, 3)
    peak_clocks = pclk.summary()

    # FP32 headline (no per-kernel events in this loop); the launch layout is
    # picked by the library's autotuner before the timed region
    f32 = torch.tensor(f64, dtype=torch.float32, device=dev)
    Q32 = torch.empty_like(f32)
    if args.no_autotune:
        p32 = make("fp32")
        tune_ms = 0.0
    else:
        # pencil layout (separable, shared, per-group) and launch layout both
        # chosen by timing on this workload
        p32, tune_ms = wke.Plan.autotuned(f32, w.d, w.N, w.L, w.n_r, w.n_s, w.n_sig, reps=3, sphere=w.sphere,
                                          precision="fp32", chunk_bytes=int(args.chunk_mb * (1 << 20)))
    tuning = wke.wke_plan_get_tuning(p32.handle)
    info = p32.info()
    with ClockSampler(dev.index) as clk:
        ms32, wall32, _ = timed(p32, f32, Q32, args.steps, args.warmup)
    clocks = clk.summary()
    # per-kernel CUDA-event timings for the roofline, in a second timed loop
    _, _, prof = timed(p32, f32, Q32, min(args.steps, 20), 1, profile=True)
    if args.fp32_only:
        line = {"metric": METRIC, "value": round(1000.0 / (sum(ms32) / len(ms32)), 3), "unit": UNIT,
                "kernels_ms": prof, "plan": {"groups_per_chunk": info.groups_per_chunk,
                                              "n_chunks": info.n_chunks},
                "tuning": {"pass2_points_per_thread": tuning.pass2_points_per_thread,
                           "pass1_units_per_block": tuning.pass1_units_per_block}, "clocks": clocks}
        p32.close()
        return line
    t_step = sum(ms32) / len(ms32)
    t_max, value = replica_rate(t_step, world, dev)

    # FP64 path on the same GPU (fewer steps: it is far slower)
    p64 = make("fp64")
    fd = torch.tensor(f64, dtype=torch.float64, device=dev)
    Q64 = torch.empty_like(fd)
    ms64, _, _ = timed(p64, fd, Q64, max(2, min(args.steps, 5)), max(1, min(args.warmup, 2)))
    fp64_rate = 1000.0 / (sum(ms64) / len(ms64))
    q32 = Q32.double().cpu().numpy()
    q64 = Q64.cpu().numpy()
    rel_err = float(np.max(np.abs(q32 - q64)) / np.max(np.abs(q64)))

    # split precision: the axis-0 transforms as TF32 tensor-core GEMMs (hi/lo split)
    psp = make("split")
    Qsp = torch.empty_like(f32)
    mssp, _, _ = timed(psp, f32, Qsp, max(3, min(args.steps, 50)), max(1, min(args.warmup, 3)))
    split = {"evals_per_s": round(1000.0 / (sum(mssp) / len(mssp)), 3),
             "rel_err_vs_fp64_gpu": float(np.max(np.abs(Qsp.double().cpu().numpy() - q64)) / np.max(np.abs(q64))),
             "what": "FP32 plan whose axis-0 DFTs run as TF32 mma.sync GEMMs with hi/lo operand splits"}
    psp.close()

    # end to end through the host-buffer call
    fh = torch.tensor(f64, dtype=torch.float32).pin_memory()
    qh = torch.empty_like(fh).pin_memory()
    wke.wke_plan_set_stream(p32.handle, stream.cuda_stream)
    for _ in range(max(1, args.warmup)):
        p32.collision_host(fh, qh)
    e2e_steps = args.steps
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        p32.collision_host(fh, qh)
    e2e_rate = world * e2e_steps / (time.perf_counter() - t0)

    # roofline of the dominant kernel class: every kernel works on chunk units
    # resident in L2 (DRAM traffic per launch is kilobytes), so the binding
    # roof is the FP32 ALU rate, measured here by the library's FMA probe
    roofline = roofline_of(prof, info, peaks32)
    fp64_info = p64.info()
    fp64_alu = {"evals_per_s": round(fp64_rate, 4), "executed_flops_per_eval": fp64_info.flops_per_collision,
                "achieved_tflops": round(fp64_info.flops_per_collision * fp64_rate / 1e12, 4),
                "peak_tflops": round(peaks64[0], 4),
                "frac": round(fp64_info.flops_per_collision * fp64_rate / 1e12 / peaks64[0], 4),
                "peak_source": "wke_alu_peak(WKE_FP64): DFMA chains on every SM, measured in this run"}

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_max, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": _config("fp32"),
        "parallelism": "replicas" if world > 1 else "single-gpu",
        "fp64_evals_per_s": round(fp64_rate, 4), "speedup_fp32_vs_fp64": round(value / world / fp64_rate, 2),
        "fp32_rel_err_vs_fp64_gpu": rel_err, "split": split, "wall_s_timed": round(wall32, 4),
        "e2e": {"value": round(e2e_rate, 3), "unit": UNIT, "h2d_bytes_per_step": fh.numel() * 4,
                "d2h_bytes_per_step": qh.numel() * 4},
        "gpu_launches": args.steps * info.launches_per_collision,
        "clocks": clocks, "roofline": roofline, "fp64_roofline": fp64_alu,
        "alu_peaks_measured": {"fp32_tflops": round(peaks32[0], 3), "fp64_tflops": round(peaks64[0], 4),
                               "sms": sms, "clocks": peak_clocks},
        "tuning": {"pass2_points_per_thread": tuning.pass2_points_per_thread,
                   "pass1_units_per_block": tuning.pass1_units_per_block,
                   "fuse_products": tuning.fuse_products, "rule_products": tuning.rule_products,
                   "layout": p32.layout or "auto", "autotune_ms": round(tune_ms, 4)},
        "plan": {"groups_per_chunk": info.groups_per_chunk, "n_chunks": info.n_chunks,
                 "separable": info.separable, "fused_products": info.fused_products,
                 "pair_planes_per_eval": info.pair_planes_per_collision, "units_per_eval": info.units_per_collision,
                 "fields_per_group": info.fields_per_group, "products_per_group": info.products_per_group,
                 "flops_per_eval": info.flops_per_collision, "l2_bytes_per_eval": info.l2_bytes_per_collision},
    }
    if args.rk:
        line["time_stepping"] = run_time_stepping(wke, torch, dev)
    if args.dealias:
        line["dealiased"] = run_dealiased(wke, torch, dev)
    if args.serve_requests > 0:
        line["serving"] = run_serving(args.serve_requests, I.BASE_SEED + 4 + rank, wke, 40 << 30, 8)
    if rank == 0 and pool is not None:
        rate, walls = cpu_oracle_rate(pool, args.oracle_evals)
        line["cpu_baseline"] = {"value": round(rate, 6), "unit": UNIT, "cores": workers, "kind": "oracle",
                                "sample": f"{len(walls)} whole evaluations of the workload (FP64 fast form, "
                                          f"node ranges over {workers} spawn processes, partial sums added "
                                          f"in node order), {sum(walls):.1f} s wall"}
    p32.close()
    p64.close()
    return line


def kernel_flops(cls, info):
    """Flops of one launch of a kernel class by the executed algorithm: 5 n
    log2 n per complex n-point transform; 16 per point for the two phase
    products and the packing of a unit in pass 1 (separable plans: 6 per
    point per row value and per pair, and 14 per point per unit for the
    axis-0 phases and packing); 30 per point per product in the per-group
    pass 2; in the product pass of the shared-field layout 12 per unit for
    the unpacking, 9 per group for s and cf, 17 per product.  A unit is two
    shifted fields packed in one transform; launch counts are averages over
    the evaluation's chunks.  With fused products the product class also
    carries the axis-0 transforms."""
    d, N = info.d, info.N_compute
    nd = N ** d
    P = nd // N
    ppg = info.products_per_group
    if info.shared_fields:
        units = info.units_per_collision / info.n_chunks
        groups = info.n_groups / info.n_chunks
    else:
        G = info.groups_per_chunk
        units = (G + 1) // 2 + G * ppg
        groups = G
    axis0 = units * P * 5.0 * N * math.log2(N) + (14.0 * units * nd if info.separable else 0.0)
    if cls == "pass1":
        if info.separable:
            # row values along axis 2 and pairs along axis 1 over every plane
            lines = (info.pair_planes_per_collision + info.row_values_per_collision) / info.n_chunks
            return lines * nd * (5.0 * math.log2(N) + 6.0)
        return units * N * (5.0 * P * math.log2(P) + 16.0 * P)
    if cls == "axis0":
        return axis0
    if cls == "pass2":
        if info.shared_fields:
            prod = nd * (12.0 * units + groups * (9.0 + 17.0 * ppg))
            return prod + (axis0 if info.fused_products else 0.0)
        per_group = (1 + ppg) * P * 5.0 * N * math.log2(N) + ppg * nd * 30.0
        return groups * per_group
    if cls == "nyquist":   # a chunk's units, two fields per transform
        return units * d * 5.0 * P * math.log2(P)
    if cls == "forward":
        return 5.0 * nd * math.log2(nd)
    return 2.0 * groups * nd


def paper_flops(cls, info):
    """Flops of one launch of a kernel class by the per-node count of the
    paper's algorithm (Sec. 3.4 complexity paragraph): per node 2 + 1/N_sig
    inverse transforms of N^d points at 5 N^d log2 N^d flops, 6 d N^d for the
    phase products and 32 N^d for the cubic products, and one forward
    transform per evaluation.  The transform's axes split between pass 1
    (the d - 1 trailing axes) and the axis-0 kernel.  The executed algorithm
    does less: it transforms each distinct shifted field once and evaluates
    each distinct product once."""
    d, N = info.d, info.N_compute
    nd = float(N) ** d
    n_sig = info.M / info.n_groups
    nodes = info.M / info.n_chunks
    fields = nodes * (2.0 + 1.0 / n_sig)
    if cls == "forward":
        return 5.0 * nd * math.log2(nd)
    if cls == "pass1":
        return fields * (5.0 * nd * math.log2(nd / N) + 6.0 * d * nd)
    if cls == "axis0":
        return fields * 5.0 * nd * math.log2(N)
    if cls == "pass2":
        prod = 32.0 * nodes * nd
        return prod if info.shared_fields else prod + fields * 5.0 * nd * math.log2(N)
    return 0.0


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch per
# kernel class, from an ncu capture of the current kernels at 3D N=64,
# M=2048, FP32 (warm L2; profiles/fused_pipeline_3d_n64_m2048_fp32.md):
# k_fused64 (interleaved unit slots) 0 + 10.2 KB, k_sep_planes64 0 + 71.4 KB.
# Remove an entry when its kernel changes after the capture.
DRAM_BYTES_3D_N64 = {"pass2": 0 + 10240, "pass1": 71424}


def roofline_of(prof, info, peak32):
    """Roofline object of the dominant kernel class (largest share of the
    serialised per-kernel CUDA-event time): executed flops per launch over the
    measured per-launch time against the measured FP32 FMA rate."""
    classes = {c: v for c, v in prof.items() if v[1] > 0}
    total = sum(v[0] for v in classes.values())
    dom = max(classes, key=lambda c: classes[c][0])
    dom_ms, dom_n = classes[dom]
    per_launch_s = dom_ms / dom_n * 1e-3
    peak = peak32[0]
    achieved = kernel_flops(dom, info) / per_launch_s / 1e12
    paper = paper_flops(dom, info) / per_launch_s / 1e12
    traffic = DRAM_BYTES_3D_N64.get(dom) if (info.d, info.N_compute, info.precision) == (3, 64, 1) else None
    return {"bound": "alu", "kernel": dom, "achieved": round(achieved, 3), "peak": round(peak, 3),
            "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": traffic,
            "peak_source": "wke_alu_peak(WKE_FP32): FMA chains on every SM, measured in this run (of measured)",
            "flops_per_launch": kernel_flops(dom, info),
            "paper_algorithm_flops_per_launch": paper_flops(dom, info),
            "paper_algorithm_achieved": round(paper, 3), "paper_algorithm_frac": round(paper / peak, 4),
            "per_launch_ms": round(dom_ms / dom_n, 5), "launches": dom_n,
            "kernel_share": {c: round(v[0] / total, 4) for c, v in classes.items()},
            "class_frac": {c: round(kernel_flops(c, info) / (v[0] / v[1] * 1e-3) / 1e12 / peak, 4)
                           for c, v in classes.items()}}


# ------------------------------------------------------------------ de-aliased variant

def run_dealiased(wke, torch, dev, reps=20):
    """3D N=32, M=1024 (16 radial x 8 x 8 cube, Gaussian with 1% noise),
    Nyquist modes zeroed: evals/s of the circular sums (N-point transforms)
    and of the de-aliased linear sums (2N = 64 grid), FP32 and FP64, CUDA
    events per evaluation with L2 flushed before each; and |sum Q| / sum |Q|
    of each FP64 result (the linear sums conserve mass exactly for this rule)."""
    w = I.WORKLOADS["3d_n32_m1024"]
    f0 = w.initial()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    out = {"workload": "3d_n32_m1024, Nyquist zeroed; de-aliased transforms on the 64^3 grid"}
    for dealias in (False, True):
        key = "dealiased" if dealias else "circular"
        res = {}
        for prec in ("fp32", "fp64"):
            plan = wke.Plan(3, w.N, w.L, w.n_r, w.n_s, w.n_sig, sphere=w.sphere, precision=prec, nyquist="zero",
                            dealias=dealias)
            f = torch.tensor(f0, dtype=plan.dtype, device=dev)
            Q = torch.empty_like(f)
            for _ in range(3):
                plan.collision(f, Q)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            for i, (a, b) in enumerate(ev):
                flush.fill_(i & 0xFF)
                a.record()
                plan.collision(f, Q)
                b.record()
            torch.cuda.synchronize()
            ms = sorted(a.elapsed_time(b) for a, b in ev)[reps // 2]
            res[f"{prec}_evals_per_s"] = round(1000.0 / ms, 3)
            if prec == "fp64":
                q = Q.cpu().numpy()
                res["mass_rel_fp64"] = float(abs(q.sum()) / abs(q).sum())
            plan.close()
        out[key] = res
    return out


# ------------------------------------------------------------------ time stepping

def run_time_stepping(wke, torch, dev):
    """RK4 on 2D N=128, M=512 (two Gaussians, 200 steps, dt = 1e-3) and RK2
    on 3D N=64, M=2048 (ring, 50 steps).  The ring's collision term reaches
    |Q| ~ 770 at max f = 1, so explicit steps of 1e-3 blow up within tens of
    steps; its run uses dt = 1e-5.  Reports steps/s (CUDA events around the
    steps; each step is one graph launch), the relative drift of mass and
    energy, and the FP32-FP64 difference after the same number of steps."""
    out = {}
    cases = [("2d_n128_m512_rk4", I.WORKLOADS["2d_n128_m512"], 4, 1e-3, 200, 200),
             ("3d_n64_m2048_rk2", WORKLOAD, 2, 1e-5, 50, 50)]
    for name, w, stages, dt, steps32, steps64 in cases:
        res, snap = {"dt": dt}, {}
        for prec, steps in (("fp64", steps64), ("fp32", steps32)):
            plan = wke.Plan(w.d, w.N, w.L, w.n_r, w.n_s, w.n_sig, sphere=w.sphere, precision=prec)
            ft = torch.tensor(w.initial(), dtype=plan.dtype, device=dev)
            m0 = plan.moments(ft).cpu().numpy()
            ms = 0.0
            done = 0
            for seg in (steps64, steps - steps64):
                if seg <= 0:
                    continue
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record()
                for _ in range(seg):
                    plan.step(ft, dt, stages)
                b.record()
                torch.cuda.synchronize()
                ms += a.elapsed_time(b)
                done += seg
                if done == steps64:
                    snap[prec] = ft.double()
            m1 = plan.moments(ft).cpu().numpy()
            res[prec] = {"steps": steps, "steps_per_s": round(steps * 1000.0 / ms, 3),
                         "mass_drift": float(abs(m1[0] - m0[0]) / abs(m0[0])),
                         "energy_drift": float(abs(m1[-1] - m0[-1]) / abs(m0[-1]))}
            plan.close()
        diff = (snap["fp32"] - snap["fp64"]).abs().max() / snap["fp64"].abs().max()
        res["fp32_vs_fp64_rel_diff_after_%d_steps" % steps64] = float(diff)
        out[name] = res
    return out


# ------------------------------------------------------------------ serving

SERVE_RATE = 200.0      # mean arrivals per second of the configured stream (Poisson)
SWEEP_RATES = (20.0, 40.0, 60.0, 80.0)


def serving_mix():
    """(d, N, n_r, n_s, n_sig) of the mixed stream: 2D N in {64, 128, 256}
    with M = 4N (N/4 x 4 x 4) and 3D N in {32, 48, 64} with M = 32N
    (N/2 x 8 x 8)."""
    return list(I.serving_request_sizes())


def _serving_initial(d, N, seed):
    if d == 2:
        return I.two_gaussians(N, 8.0, seed)
    return I.ring(3, N, 8.0) if seed % 2 else I.gaussian_noise(3, N, 8.0, seed)


def shape_step_ms(wke, seed):
    """Milliseconds of one FP32 RK4 step (dt = 1e-3) of every request shape
    of the mix, each run alone on the GPU (CUDA events, 2 warm-up and 5 timed
    steps; the plans the server would build)."""
    import torch
    out = {}
    for d, N, n_r, n_s, n_sig in serving_mix():
        plan = wke.Plan(d, N, 8.0, n_r, n_s, n_sig, precision="fp32")
        f0 = torch.tensor(_serving_initial(d, N, seed), dtype=torch.float32, device="cuda")
        f = f0.clone()
        for _ in range(2):
            plan.step(f, 1e-3, 4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f.copy_(f0)
        e0.record()
        for _ in range(5):
            plan.step(f, 1e-3, 4)
        e1.record()
        torch.cuda.synchronize()
        out[(d, N)] = e0.elapsed_time(e1) / 5
        plan.close()
    return out


def run_stream(n_requests, seed, rate, wke, budget_bytes, max_active, step_ms=None):
    """A seeded Poisson stream at `rate` req/s of mixed requests (1-20 RK4
    steps, dt = 1e-3, FP32) through the continuous-batching server; latency
    is completion minus submission on the server's clock.  With `step_ms`
    (shape_step_ms) it also reports the stream's serial GPU time: every
    request's steps timed alone and added up, over the stream's wall time,
    and the share of that time in 2D requests."""
    import numpy as np
    sizes = serving_mix()
    u = I.splitmix64_uniform(seed, 3 * n_requests)
    gaps = -np.log(1.0 - u[0::3]) / rate
    arrive = np.cumsum(gaps)
    reqs = []
    for k in range(n_requests):
        d, N, n_r, n_s, n_sig = sizes[int(u[3 * k + 1] * len(sizes))]
        steps = 1 + int(u[3 * k + 2] * 20)
        reqs.append((d, N, n_r, n_s, n_sig, steps, _serving_initial(d, N, seed + k).astype(np.float32)))
    srv = wke.Server(device_budget_bytes=budget_bytes, max_active=max_active)
    try:
        # one request of every shape first (not timed), so that plan creation
        # does not count as latency of the measured stream
        warm = [srv.submit(r[6], r[2], r[3], r[4], 1, 1e-3)[0] for r in
                {(r[0], r[1]): r for r in reqs}.values()]
        for w_id in warm:
            srv.wait(w_id, timeout_s=600)
        t0 = time.perf_counter()
        ids = []
        for k, (d, N, n_r, n_s, n_sig, steps, f) in enumerate(reqs):
            delay = arrive[k] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit(f, n_r, n_s, n_sig, steps, 1e-3)[0])
        stats = [srv.wait(i, timeout_s=600) for i in ids]
    finally:
        srv.close()
    ok = [st for st in stats if st.status == wke.WKE_OK]
    lat = np.array([st.t_done - st.t_submit for st in ok]) * 1000.0
    wait = np.array([st.t_admit - st.t_submit for st in ok]) * 1000.0
    span = max(st.t_done for st in ok) - min(st.t_submit for st in ok)
    evals = sum(4 * r[5] for r in reqs)
    out = {"offered_req_s": rate, "requests": n_requests, "completed": len(ok),
           "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
           "admission_wait_p50_ms": round(float(np.percentile(wait, 50)), 3),
           "served_req_s": round(len(ok) / span, 3), "q_evals_per_s": round(evals / span, 2)}
    if step_ms:
        serial = [r[5] * step_ms[(r[0], r[1])] for r in reqs]
        out["serial_gpu_s_over_wall"] = round(sum(serial) / 1000.0 / span, 3)
        out["serial_share_2d"] = round(sum(t for t, r in zip(serial, reqs) if r[0] == 2) / sum(serial), 4)
    return out


def run_serving(n_requests, seed, wke, budget_bytes, max_active):
    """Latency and throughput of the mixed stream at offered loads below and
    at saturation (SWEEP_RATES) and at the configured SERVE_RATE; the served
    rate at SERVE_RATE is the saturation throughput."""
    step_ms = shape_step_ms(wke, seed)
    sweep = [run_stream(n_requests, seed + 1000 * i, rate, wke, budget_bytes, max_active, step_ms)
             for i, rate in enumerate(SWEEP_RATES)]
    cfg = run_stream(n_requests, seed, SERVE_RATE, wke, budget_bytes, max_active, step_ms)
    return {"sweep": sweep, "configured": cfg, "saturation_req_s": cfg["served_req_s"],
            "rk4_step_ms_alone": {f"{d}d_n{N}": round(v, 4) for (d, N), v in step_ms.items()},
            "max_active": max_active, "budget_gib": round(budget_bytes / 2 ** 30, 1),
            "latency": "submission to completion on the server clock; one plan of every shape created before "
                       "each stream",
            "mix": "2D N in {64,128,256} (M=4N), 3D N in {32,48,64} (M=32N); steps U{1..20} RK4, dt=1e-3, FP32"}


# ------------------------------------------------------------------ reference arm

def run_reference(args, rank, world):
    """The reference arm: the CPU FP64 oracle (the only other program that
    computes this operator), one whole evaluation of the workload per step
    over the host cores.  The warm-up steps evaluate the nodes of one radius
    each (they start the worker processes and their imports)."""
    if rank != 0:
        return None
    from oracle import wke_oracle as O
    pool, workers = make_pool()
    w = WORKLOAD
    f = w.initial()
    qa = _oracle_quad_args()
    try:
        for _ in range(args.warmup):
            pool.collision_fast(f, w.L, (qa[0], 1) + qa[2:])
        walls = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            walls.append(pool.collision_fast(f, w.L, qa)[1])
        wall = time.perf_counter() - t0
    finally:
        pool.close()
    del O
    ms = 1000.0 * sum(walls) / len(walls)
    rate = 1000.0 / ms
    return {"impl": "reference", "metric": METRIC, "value": round(rate, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config("fp64 (CPU oracle)"),
            "cpu_baseline": {"value": round(rate, 6), "unit": UNIT, "cores": workers, "kind": "oracle",
                             "sample": f"{args.steps} whole evaluation{'s' if args.steps != 1 else ''}, one per step, node ranges over "
                                       f"{workers} spawn processes; {wall:.1f} s wall"},
            "e2e": {"value": round(rate, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--oracle-evals", type=int, default=2,
                    help="whole oracle evaluations timed for the CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch layout")
    ap.add_argument("--no-rk", dest="rk", action="store_false", help="skip the time-stepping section")
    ap.add_argument("--no-dealias", dest="dealias", action="store_false",
                    help="skip the de-aliased-variant section")
    ap.add_argument("--serve-requests", type=int, default=80,
                    help="requests in each serving stream (0: skip serving)")
    ap.add_argument("--fp32-only", action="store_true",
                    help="only the FP32 timing and kernel split (profiling runs)")
    ap.add_argument("--chunk-mb", type=float, default=0.0,
                    help="intermediate-field budget per chunk in MiB (0: library default)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line:
            print(json.dumps(line), flush=True)
        return
    # the oracle's process pool starts before the first GPU call
    pool, workers = (None, 0)
    if rank == 0 and not (args.no_cpu_baseline or args.fp32_only):
        pool, workers = make_pool()
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    try:
        line = run_gpu(args, rank, world, pool, workers)
    finally:
        if pool is not None:
            pool.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
