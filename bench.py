"""Benchmark of the ALI hot path on synthetic inputs shaped like the paper's models.

A step is one accelerated Lambda iteration on the 3D clumpy cloud (50k points, 48 HEALPix
rays = 24 ray pairs, 5-level rotor with 4 lines x 31 Gauss-Hermite bins): line data ->
Feautrier formal solve of every (point, ray pair, bin) -> statistical equilibrium ->
convergence measure. The rays are traced once before the timed region (the mesh is
static across iterations, Sec. 3.2).

metric: point-ray-pair-frequency Feautrier solves per second (whole job).
value : device-resident inputs, CUDA events around K steps on the library's stream.
e2e   : the same steps through the C ABI with host buffers: populations copied in from
        pinned memory and read back every step.
Multi-GPU (torchrun): every rank solves its own independently seeded model; no
collective on the data path (weak scaling); max time over ranks.

--impl reference times the FP64 CPU oracle on host cores on a bounded sample of the
same workload (the reference arm: there is no other implementation to run).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = dict(workload="3D clumpy cloud, 50k points, k=16 symmetric NN, 48 rays (HEALPix nside=2), "
                         "5-level linear rotor, 4 lines x 31 Gauss-Hermite bins, radial outflow to 10 km/s",
                n_points=50_000, n_rays=48, n_lines=4, n_bins=31)
METRIC = "point-ray-pair-frequency Feautrier solves/s"
UNIT = "solves/s"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mg_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1])); mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        try:
            os.remove(self.path)
        except OSError:
            pass
        return out


def reduce_max(values, device="cpu"):
    """Element-wise maximum of per-rank timings over all ranks (identity for one rank)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def whole_job_rate(units_per_rank, steps, world_size, ms_max):
    """Units processed by all ranks divided by the slowest rank's time (weak scaling:
    every rank solves its own model)."""
    return world_size * units_per_rank * steps / (ms_max * 1e-3)


def build_model(seed):
    import synthetic as syn
    return syn.model_clumpy_3d(n=WORKLOAD["n_points"], seed=seed)


def recorded_traffic(kernel_variant):
    """DRAM bytes per launch of the formal-solve kernel from the committed ncu record,
    used only while the kernel's source is unchanged since the capture (else None)."""
    import hashlib
    rec_p = os.path.join(ROOT, "profiles", "feautrier_warp_clumpy50k.json")
    if not os.path.exists(rec_p):
        return None
    rec = json.load(open(rec_p))
    src = os.path.join(ROOT, rec["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != rec["source_sha256"]:
        return None
    if kernel_variant != rec.get("variant"):      # the record belongs to one launch variant
        return None
    return rec["dram_bytes_read_per_launch"] + rec["dram_bytes_write_per_launch"]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ oracle (CPU) timing
def time_oracle(model, target_s=15.0, seed=0):
    """Times the FP64 oracle's formal solve on a bounded sample of origin points, grown
    until it takes about target_s seconds; returns solves/s, threads and the sample."""
    from oracle import Oracle
    threads = os.cpu_count() or 1
    o = Oracle(model, nthreads=threads)
    pops = o.lte()
    rng = np.random.default_rng(seed)
    P = o.dirs.shape[0] // 2
    F = model.species.n_lines * o.Q
    k = 16
    while True:
        origins = np.sort(rng.choice(model.n, k, replace=False))
        t0 = time.perf_counter()
        o.formal_solve(pops, origins)
        dt = time.perf_counter() - t0
        if dt > target_s / 4 or k >= model.n:
            break
        k = min(model.n, int(k * max(2.0, target_s / 4 / max(dt, 1e-3))))
    solves = k * P * F
    return solves / dt, threads, f"{k} of {model.n} origin points ({solves} solves, {dt:.1f} s)"


def time_oracle_one_thread(model, target_s=5.0, seed=1):
    """The same oracle timing on one host thread (a smaller sample)."""
    from oracle import Oracle
    o = Oracle(model, nthreads=1)
    pops = o.lte()
    rng = np.random.default_rng(seed)
    P = o.dirs.shape[0] // 2
    F = model.species.n_lines * o.Q
    k = 2
    while True:
        origins = np.sort(rng.choice(model.n, k, replace=False))
        t0 = time.perf_counter()
        o.formal_solve(pops, origins)
        dt = time.perf_counter() - t0
        if dt > target_s / 4 or k >= model.n:
            break
        k = min(model.n, int(k * max(2.0, target_s / 4 / max(dt, 1e-3))))
    return k * P * F / dt, f"{k} origin points, 1 thread, {dt:.1f} s"


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch
    import torch.distributed as dist
    import paper_1912_08445_gb300 as mg

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    model = build_model(seed=rank)
    prec = mg.MG_MIXED if args.precision == "mixed" else mg.MG_FP64
    ctx = mg.Context(device=local, precision=prec, profile=0)
    ctx.set_stream(stream.cuda_stream)
    ctx.load_model(model)
    st, _ = ctx.trace_rays()
    ctx.init_populations()
    tuned = ctx.autotune(reps=2) if prec == mg.MG_MIXED else (-1, None, 0)
    solves, updates = ctx.work_counts()
    n, lev = model.n, model.species.n_lev

    def step():
        ctx.formal_solve()
        ctx.update_populations()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        clocks = Clocks(local)
        clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        clk = clocks.stop()

        # per-kernel times of the dominant kernel (events on the same stream)
        ctx.close()
        ctx = mg.Context(device=local, precision=prec, profile=1)
        ctx.set_stream(stream.cuda_stream)
        ctx.load_model(model)
        ctx.trace_rays()
        ctx.init_populations()
        ctx.set_variant(tuned[0])
        step()
        ctx.reset_kernel_times()
        for _ in range(max(2, min(args.steps, 5))):
            step()
        kt = ctx.kernel_times()

        # end to end through the C ABI with pinned host buffers
        h_in = torch.empty((n, lev), dtype=torch.float64, pin_memory=True).numpy()
        h_out = torch.empty((n, lev), dtype=torch.float64, pin_memory=True).numpy()
        h_in[:] = ctx.get_populations()
        for _ in range(2):
            ctx.set_populations(h_in); step(); ctx.get_populations(out=h_out)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.set_populations(h_in)
            step()
            ctx.get_populations(out=h_out)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0

    ms_max, e2e_ms_max = reduce_max([ms, e2e_s * 1e3], device=f"cuda:{local}")
    if ws > 1:
        dist.barrier()

    if rank == 0:
        pk, pk_kind = peaks()
        kname = "feautrier_mixed" if prec == mg.MG_MIXED else "feautrier_fp64"
        k_ms, k_n = kt.get(kname, (float("nan"), 1))
        k_avg = k_ms / max(k_n, 1)
        # algorithmic work of one formal-solve launch: cell-frequency updates x flops per
        # update (FP32: 16 FMA-pipe flops + 2 MUFU ops; FP64: 18 flops, exp and divide
        # counted as one each)
        flops_per_update = 18.0
        if prec == mg.MG_MIXED:
            peak = 152 * 128 * 2 * 2.07e9 / 1e12
            peak_note = "FP32 FMA lanes x 2 x 2.07 GHz (derived)"
        else:
            peak = 1.25
            peak_note = "nominal FP64 1.25 TFLOP/s (GB300)"
        achieved = updates * flops_per_update / (k_avg * 1e-3) / 1e12
        traffic = recorded_traffic(tuned[0]) if prec == mg.MG_MIXED else None
        roof = {"bound": "alu", "achieved": round(achieved, 4), "peak": peak, "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": kname,
                "kernel_ms": round(k_avg, 3), "peak_source": peak_note,
                "cell_freq_updates_per_launch": updates,
                "hbm_algorithmic_GBps": round(st["n_elements"] * 16 / (k_avg * 1e-3) / 1e9, 2),
                "hbm_algorithmic_frac_of_measured": round(st["n_elements"] * 16 / (k_avg * 1e-3) / 1e9 / pk["hbm_gbs"], 5)}
        cpu_v, cores, sample = time_oracle(model) if args.cpu_baseline else (None, None, None)
        cpu_1 = time_oracle_one_thread(model) if args.cpu_baseline else None
        value = whole_job_rate(solves, args.steps, ws, ms_max)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == mg.MG_MIXED else "f64", "data": "synthetic",
            "config": dict(WORKLOAD, precision=args.precision, l2="inputs larger than L2 (ray store "
                           f"{st['n_elements'] * 24 / 1e9:.2f} GB read per step)",
                           parallelism=f"replicas x{ws}", solves_per_step=solves,
                           cell_freq_updates_per_step=updates, mean_pair_len=round(st["mean_pair_len"], 1),
                           launch_variant=tuned[0], variants_tried=tuned[2]),
            "e2e": {"value": whole_job_rate(solves, args.steps, ws, e2e_ms_max), "unit": UNIT,
                    "h2d_bytes_per_step": n * lev * 8, "d2h_bytes_per_step": n * lev * 8},
            "gpu_launches": 3 * args.steps,
            "clocks": clk,
            "roofline": roof,
            "cpu_baseline": None if cpu_v is None else {"value": cpu_v, "unit": UNIT, "cores": cores,
                                                        "kind": "oracle", "sample": sample,
                                                        "single_thread": {"value": cpu_1[0], "unit": UNIT,
                                                                          "sample": cpu_1[1]}},
            "peaks_source": pk_kind,
        }
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    model = build_model(seed=0)
    from oracle import Oracle
    threads = os.cpu_count() or 1
    o = Oracle(model, nthreads=threads)
    pops = o.lte()
    P = o.dirs.shape[0] // 2
    F = model.species.n_lines * o.Q
    k = 256
    rng = np.random.default_rng(0)
    origins = np.sort(rng.choice(model.n, k, replace=False))
    for _ in range(args.warmup):
        o.formal_solve(pops, origins[:32])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        J, L, E = o.formal_solve(pops, origins)
    dt = time.perf_counter() - t0
    solves = k * P * F * args.steps
    v = solves / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(WORKLOAD, precision="fp64"),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{k} of {model.n} origin points per step ({k * P * F} solves)"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------ ALI time to converge
def run_ali(args):
    """ALI time-to-converge on the workload: from LTE populations to a max relative change
    below 1e-6, for each requested precision, with Ng off and on. Rays are traced once
    beforehand (not timed); the timed region is the whole iteration loop."""
    import torch
    import paper_1912_08445_gb300 as mg
    model = build_model(seed=0)
    stream = torch.cuda.Stream()
    out = {"metric": "ALI time to converge (max relative population change < 1e-6)", "unit": "s",
           "higher_is_better": False, "data": "synthetic", "config": dict(WORKLOAD), "runs": []}
    for prec_name in args.ali_precisions.split(","):
        prec = mg.MG_MIXED if prec_name == "mixed" else mg.MG_FP64
        for ng in (0, 4):
            ctx = mg.Context(precision=prec, tol=1e-6, max_iter=args.ali_max_iter, ng_period=ng)
            ctx.set_stream(stream.cuda_stream)
            ctx.load_model(model)
            torch.cuda.synchronize()
            t_tr = time.perf_counter()
            ctx.trace_rays()
            torch.cuda.synchronize()
            trace_s = time.perf_counter() - t_tr
            ctx.init_populations()
            if prec == mg.MG_MIXED:
                ctx.autotune(reps=1)
                ctx.init_populations()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep, rc = ctx.iterate(allow_not_converged=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            out["runs"].append({"precision": prec_name, "ng_period": ng, "seconds": dt,
                                "iterations": rep["iterations"], "ng_steps": rep["ng_steps"],
                                "converged": bool(rep["converged"]), "last_change": rep["last_change"],
                                "fallback_cells": rep["n_fallback"], "trace_seconds_untimed": trace_s})
            ctx.close()
    print(json.dumps(out))


# ------------------------------------------------------------------ other configurations
def run_batch(args):
    """Batched models: 64 independent clumpy clouds of 2k-40k points (seeded log-uniform
    sizes, per-model outflow speeds so that ray lengths span ~10-400 points), mixed
    precision. Reports the batched formal solve (one persistent launch after the line data
    of every model) against a loop of per-model launches, and the batched ALI to 1e-6."""
    import torch
    import paper_1912_08445_gb300 as mg
    import synthetic as syn
    t0 = time.perf_counter()
    models = syn.model_batch(seed=3, n_models=args.batch_models)
    gen_s = time.perf_counter() - t0
    ctxs = []
    for m in models:
        c = mg.Context(precision=mg.MG_MIXED, tol=1e-6, max_iter=100, ng_period=0)
        c.load_model(m)
        c.trace_rays()
        c.init_populations()
        ctxs.append(c)
    b = mg.Batch(ctxs)
    v, srt, tune_ms = b.autotune(reps=2)
    solves, updates = b.work_counts()
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        b.formal_solve()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b.formal_solve()
    torch.cuda.synchronize()
    batched = (time.perf_counter() - t0) / args.steps
    for c in ctxs:
        c.set_variant(v)
    for _ in range(args.warmup):
        for c in ctxs:
            c.formal_solve()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for c in ctxs:
            c.formal_solve()
    torch.cuda.synchronize()
    looped = (time.perf_counter() - t0) / args.steps
    for c in ctxs:
        c.init_populations()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps, rc = b.iterate(allow_not_converged=True)
    ali_s = time.perf_counter() - t0
    its = [r["iterations"] for r in reps]
    print(json.dumps({
        "metric": METRIC, "unit": UNIT, "workload": f"{len(models)} clumpy clouds, "
        f"{min(m.n for m in models)}-{max(m.n for m in models)} points, 48 rays, 4 lines x 31 bins",
        "points_total": int(sum(m.n for m in models)), "solves_per_formal_solve": solves,
        "cell_freq_updates": updates, "batched_value": solves / batched, "batched_ms": batched * 1e3,
        "looped_value": solves / looped, "looped_ms": looped * 1e3, "variant": v, "queue_sorted": srt,
        "ali_seconds": ali_s, "ali_iterations_min_max": [min(its), max(its)],
        "ali_converged": int(sum(r["converged"] for r in reps)), "generation_s": gen_s}))


def run_disc(args):
    """Keplerian disc (200k points, 192 rays, 20-level rotor, 19 lines x 63 bins), mixed
    precision: one ALI iteration per step. With --tau-fp64 T the cells whose diagonal ALO
    weight reaches 1 - 1/T are solved again in FP64 every step."""
    import numpy as np
    import torch
    import paper_1912_08445_gb300 as mg
    import synthetic as syn
    m = syn.model_disc(n=args.disc_points, seed=0)
    ctx = mg.Context(precision=mg.MG_MIXED, profile=1, tau_fp64=args.tau_fp64)
    ctx.load_model(m)
    t0 = time.perf_counter()
    st, _ = ctx.trace_rays()
    trace_s = time.perf_counter() - t0
    ctx.init_populations()
    v, tms, nt = ctx.autotune(reps=1)
    solves, updates = ctx.work_counts()
    ctx.reset_kernel_times()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.formal_solve()
        ctx.update_populations()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    kt = ctx.kernel_times()
    ctx.formal_solve()   # (untimed) the radiation field of the final populations, for max L
    max_L = float(np.max(ctx.get_radiation()[1]))
    print(json.dumps({"metric": METRIC, "unit": UNIT, "workload": "Keplerian disc, "
                      f"{m.n} points, 192 rays, 20 levels, 19 lines x 63 bins", "value": solves / dt,
                      "ms_per_step": dt * 1e3, "cell_freq_updates": updates, "variant": v,
                      "tau_fp64": args.tau_fp64, "promoted_cells": ctx.promoted_cells() if args.tau_fp64 > 0 else 0,
                      "max_L": max_L,
                      "trace_s": trace_s, "ray_stats": st, "kernel_ms": {k: v2[0] / max(v2[1], 1) for k, v2 in kt.items()}}))


def run_image(args):
    """Images of the Keplerian disc (Sec. 3.5): one image per step of the lowest line
    along one ray direction, 63 channels over +-15 km/s, every point a pixel; FP32 in a
    mixed-precision context, and FP64 in an FP64 context.
    value: pixel-channel intensities per second from the image kernel's CUDA-event time;
    e2e: the same through mg_image with the image copied back to host memory every step.
    The algorithmic work (points of the pairs along that direction x channels) is
    estimated from 4000 sampled pairs."""
    import numpy as np
    import torch
    import paper_1912_08445_gb300 as mg
    import synthetic as syn
    m = syn.model_disc(n=args.disc_points, seed=0)
    ray, n_ch = 40, 63
    u = np.linspace(-15e3, 15e3, n_ch)
    pix = m.n * n_ch
    imgs = {}
    out = {"metric": "image pixel-channel intensities/s", "unit": "intensities/s",
           "workload": f"Keplerian disc, {m.n} points, image along ray {ray} of 192, line 0, "
                       f"{n_ch} channels over +-15 km/s"}
    for prec, kname in ((mg.MG_MIXED, "image_fp32"), (mg.MG_FP64, "image_fp64")):
        ctx = mg.Context(precision=prec, profile=1)
        ctx.load_model(m)
        ctx.trace_rays()
        ctx.init_populations()
        if "mean_pair_points" not in out:
            anti = ctx.get_directions()[1][ray]
            samp = np.random.default_rng(0).choice(m.n, min(4000, m.n), replace=False)

            def half_points(o, r):
                g = ctx.get_ray(int(o), r, cap=8192)
                return len(g["cells"]) + int(g["nsub"].sum())
            out["mean_pair_points"] = float(np.mean([1 + half_points(o, ray) + half_points(o, anti) for o in samp]))
        updates = out["mean_pair_points"] * pix
        dI = torch.empty((m.n, n_ch), dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            ctx.image_dev(ray, 0, u, dI.data_ptr())
        ctx.reset_kernel_times()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            ctx.image_dev(ray, 0, u, dI.data_ptr())
        torch.cuda.synchronize()
        k_ms, k_n = ctx.kernel_times()[kname]
        kernel_s = k_ms / k_n / 1e3
        t0 = time.perf_counter()
        for _ in range(args.steps):
            I, xy = ctx.image(ray, 0, u)
        e2e_s = (time.perf_counter() - t0) / args.steps
        rec = {"value": pix / kernel_s, "ms_per_image": kernel_s * 1e3,
               "e2e": {"value": pix / e2e_s, "unit": "intensities/s", "ms_per_image": e2e_s * 1e3,
                       "d2h_bytes_per_step": int(pix * 8 + m.n * 16)},
               "cell_channel_updates_per_s": updates / kernel_s, "max_I": float(I.max()), "min_I": float(I.min())}
        imgs[prec] = I
        if prec == mg.MG_FP64:
            # FP64 bound per point-channel update at the measured pipe rates of this GPU: three
            # exponentials (profile, exp(-dtau), expm1), two divisions, ~30 DFMA-pipe operations
            bound_s = updates * (3 / 31e9 + 2 / 66e9 + 30 / 0.50e12)
            rec.update(fp64_bound_ms=bound_s * 1e3, fraction_of_fp64_bound=bound_s / kernel_s)
            out["fp64"] = rec
        else:
            out["fp32"] = rec
            out["value"] = rec["value"]
        ctx.close()
        del dI
    a, b = imgs[mg.MG_MIXED], imgs[mg.MG_FP64]
    out["fp32_vs_fp64_max_rel_diff"] = float(np.max(2 * np.abs(a - b) / (np.abs(a) + np.abs(b))))
    print(json.dumps(out))


def run_sphere1d(args):
    """1D spherically symmetric cloud (200 log-spaced shells, 2-level species, 12 rays,
    31 bins, FP64): formal-solve throughput of one ALI step, and the ALI from LTE to a
    1e-6 relative change (Ng off and on) on the GPU and with the FP64 oracle on the host
    cores (all threads and one thread), with the converged populations compared."""
    import numpy as np
    import torch
    import paper_1912_08445_gb300 as mg
    import synthetic as syn
    from oracle import Oracle
    m = syn.model_sphere_1d(n=200, seed=0)
    threads = os.cpu_count() or 1
    out = {"metric": "ALI time to converge (max relative population change < 1e-6)", "unit": "s",
           "workload": "1D spherical cloud, 200 shells, 2-level species, 12 rays (nside=1), 1 line x 31 bins, FP64",
           "runs": []}
    ctx = mg.Context(precision=mg.MG_FP64, profile=1)
    ctx.load_model(m)
    ctx.trace_rays()
    ctx.init_populations()
    solves, updates = ctx.work_counts()
    for _ in range(args.warmup):
        ctx.formal_solve()
        ctx.update_populations()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.formal_solve()
        ctx.update_populations()
    torch.cuda.synchronize()
    step_s = (time.perf_counter() - t0) / args.steps
    out["solves_per_step"] = solves
    out["gpu_solves_per_s"] = solves / step_s
    out["gpu_ms_per_step"] = step_s * 1e3
    ctx.close()
    o_all = Oracle(m, nthreads=threads)
    o_one = Oracle(m, nthreads=1)
    for ng in (0, 4):
        c = mg.Context(precision=mg.MG_FP64, tol=1e-6, max_iter=400, ng_period=ng)
        c.load_model(m, dirs=o_all.dirs)
        c.trace_rays()
        c.init_populations()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep, rc = c.iterate(allow_not_converged=True)
        torch.cuda.synchronize()
        gpu_s = time.perf_counter() - t0
        pops = c.get_populations()
        c.close()
        rec = {"ng_period": ng, "gpu_seconds": gpu_s, "gpu_iterations": rep["iterations"],
               "gpu_converged": bool(rep["converged"])}
        for name, o in (("oracle", o_all), ("oracle_1thread", o_one)):
            t0 = time.perf_counter()
            ref, ch, conv = o.ali(tol=1e-6, max_iter=400, ng_period=ng)
            rec[name + "_seconds"] = time.perf_counter() - t0
            rec[name + "_iterations"] = len(ch)
        rec["max_rel_diff_gpu_vs_oracle"] = float(np.max(2 * np.abs(pops - ref) / (np.abs(pops) + np.abs(ref))))
        out["runs"].append(rec)
    out["oracle_threads"] = threads
    print(json.dumps(out))


def run_learned(args):
    """Learned initial populations (20-level rotor): trains the network on converged
    populations of seeded cloud/disc models, then compares on held-out seeds the ALI to
    1e-6 from the network's start (mixed precision) with the LTE start (mixed) and with
    the plain FP64 ALI from LTE, on the same GPU (Ng off and on)."""
    import numpy as np
    import torch
    import paper_1912_08445_gb300 as mg
    import synthetic as syn
    from paper_1912_08445_gb300 import learned
    sp = syn.species_rotor(20, np.random.default_rng(77))
    t0 = time.perf_counter()
    train = learned.corpus_models(args.corpus, 1000, n_points=args.corpus_points, species=sp)
    X, Y, reps = learned.build_corpus(train, ng_period=4)
    corpus_s = time.perf_counter() - t0
    net, trep = learned.train_network(X, Y, 20, epochs=args.epochs, batch=4096, lr=2e-3)
    held = learned.corpus_models(10, 5000, n_points=args.corpus_points, species=sp)
    rows = []
    for m in held:
        for ng in (0, 4):
            rec = {"n": m.n, "shape": m.name, "ng_period": ng}
            for name, prec, start in (("fp64_lte", mg.MG_FP64, "lte"), ("mixed_lte", mg.MG_MIXED, "lte"),
                                      ("mixed_mlp", mg.MG_MIXED, "mlp")):
                ctx = mg.Context(precision=prec, tol=1e-6, max_iter=400, ng_period=ng)
                ctx.load_model(m)
                ctx.trace_rays()
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                if start == "lte":
                    ctx.init_populations()
                else:
                    ctx.init_populations_mlp(net)
                rep, rc = ctx.iterate(allow_not_converged=True)
                torch.cuda.synchronize()
                rec[name] = {"seconds": time.perf_counter() - t1, "iterations": rep["iterations"],
                             "converged": bool(rep["converged"])}
                ctx.close()
            rows.append(rec)
    summ = {}
    for ng in (0, 4):
        sel = [r for r in rows if r["ng_period"] == ng]
        for name in ("fp64_lte", "mixed_lte", "mixed_mlp"):
            summ[f"{name}_ng{ng}"] = {"mean_seconds": float(np.mean([r[name]["seconds"] for r in sel])),
                                      "mean_iterations": float(np.mean([r[name]["iterations"] for r in sel])),
                                      "all_converged": all(r[name]["converged"] for r in sel)}
    print(json.dumps({"metric": "ALI time to converge (1e-6), held-out seeds", "unit": "s", "higher_is_better": False,
                      "workload": f"20-level rotor, cloud/disc models of {args.corpus_points} points, 48 rays, 19 lines x 31 bins",
                      "corpus_models": len(train), "corpus_rows": int(X.shape[0]), "corpus_seconds": corpus_s,
                      "training": trep, "summary": summ, "runs": rows}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--ali", action="store_true", help="measure ALI time to converge instead")
    ap.add_argument("--workload", default="clumpy", choices=["clumpy", "batch", "disc", "learned", "image", "sphere1d"])
    ap.add_argument("--corpus", type=int, default=200)
    ap.add_argument("--corpus-points", type=int, default=3000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch-models", type=int, default=64)
    ap.add_argument("--disc-points", type=int, default=200_000)
    ap.add_argument("--tau-fp64", type=float, default=0.0,
                    help="disc workload: re-solve cells with L >= 1 - 1/T in FP64 (0: off)")
    ap.add_argument("--ali-precisions", default="mixed")
    ap.add_argument("--ali-max-iter", type=int, default=300)
    args = ap.parse_args()
    if args.workload == "batch":
        run_batch(args)
    elif args.workload == "disc":
        run_disc(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "image":
        run_image(args)
    elif args.workload == "sphere1d":
        run_sphere1d(args)
    elif args.ali:
        run_ali(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
