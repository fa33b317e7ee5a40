"""Benchmark of the ALI hot path on synthetic inputs shaped like the paper's models.

Default line (the headline): the Keplerian disc -- 200k points in a flared disc, 192
HEALPix rays (96 ray pairs), a 20-level linear rotor with 19 lines x 63 Gauss-Hermite
bins -- dense enough that the line-centre optical depth of the low lines reaches ~1e4, in
mixed precision: the FP32 formal solve with the cancellation-free elimination, FP64
statistical equilibrium. A step is one accelerated Lambda iteration: line data ->
Feautrier formal solve of every (point, ray pair, bin) -> statistical equilibrium ->
convergence measure. The rays are traced once before the timed region (the mesh is
static across iterations, Sec. 3.2).
fp64_elimination: the same construction at 10k points, one step with the cells of
optical depth above 1e2 (diagonal ALO weight >= 0.99) solved again in FP64, against the
FP32 step: promoted share, time, and how far the FP32 results were from the FP64 ones.

metric: point-ray-pair-frequency Feautrier solves per second (whole job).
value : device-resident inputs, CUDA events around K steps on the library's stream.
e2e   : the same steps through the C ABI with host buffers: populations copied in from
        pinned memory and read back every step.
ali   : the second half of the metric, in the same run: ALI time to converge (max relative
        population change < 1e-6) on the 3D clumpy cloud (50k points, 48 rays, 5-level
        rotor, 4 lines x 31 bins): plain FP64 from LTE, mixed from LTE, and mixed from
        the populations of a network trained in the run on converged clouds of the same
        species (held-out seeds), each with Ng off and on.
Multi-GPU (torchrun): every rank solves its own independently seeded model; no
collective on the data path (weak scaling); max time over ranks.

--impl reference times the FP64 CPU oracle on host cores on a bounded sample of the
disc (the reference arm: there is no other implementation to run).
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

DISC_N_H2_IN = 2.5e16   # n_H2 at the inner radius (m^-3): line-centre optical depths ~1e4
DISC_TAU_FP64 = 100.0
WORKLOAD = dict(workload="Keplerian disc, 200k points (flared, n ~ r^-1 exp(-z^2/2H^2), H/r = 0.1, T ~ r^-0.5, "
                         "Keplerian velocity around 1 M_sun), 192 rays (HEALPix nside=4), 20-level linear rotor, "
                         "19 lines x 63 Gauss-Hermite bins, line-centre optical depths up to ~1e4",
                n_points=200_000, n_rays=192, n_lines=19, n_bins=63, n_h2_in=DISC_N_H2_IN)
CLUMPY = dict(workload="3D clumpy cloud, 50k points, k=16 symmetric NN, 48 rays (HEALPix nside=2), "
                       "5-level linear rotor, 4 lines x 31 Gauss-Hermite bins, radial outflow to 10 km/s",
              n_points=50_000, n_rays=48, n_lines=4, n_bins=31)
METRIC = "point-ray-pair-frequency Feautrier solves/s"
UNIT = "solves/s"
# One point-bin update of the FP32 sweep: 11 FP32 operations on the FMA pipe (FMA, MUL or
# ADD, one each: profile argument, square, line opacity, floored source, dtau, t, Phi,
# 1 + dtau Phi, psi), of which 4 are FMAs (15 flops with FMA = 2); one ex2 and one rcp.
FMA_OPS_PER_UPDATE = 11.0
FLOPS_PER_UPDATE = 15.0
MUFU_PER_UPDATE = (1, 1)  # ex2, rcp per point-bin update


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
        with open(self.path) as f:
            out = self.parse(f) or out
        try:
            os.remove(self.path)
        except OSError:
            pass
        return out

    @staticmethod
    def parse(lines):
        """Median SM clock, maximum clock and the throttle reasons seen in nvidia-smi CSV
        lines of the query above (None without a valid sample)."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
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
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


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
    return syn.model_disc(n=WORKLOAD["n_points"], seed=seed, n_h2_in=DISC_N_H2_IN)


def build_clumpy(seed):
    import synthetic as syn
    return syn.model_clumpy_3d(n=CLUMPY["n_points"], seed=seed)


def recorded_traffic(kernel_variant, record="feautrier_warp_disc200k.json", root=ROOT):
    """DRAM bytes per launch of the formal-solve kernel from the committed ncu record,
    used only while the kernel's source is unchanged since the capture (else None)."""
    import hashlib
    rec_p = os.path.join(root, "profiles", record)
    if not os.path.exists(rec_p):
        return None
    rec = json.load(open(rec_p))
    src = os.path.join(root, rec["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != rec["source_sha256"]:
        return None
    cap = rec.get("captures", {}).get(str(kernel_variant))   # one capture per launch variant
    if cap is None:
        return None
    return cap["dram_bytes_read_per_launch"] + cap["dram_bytes_write_per_launch"]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ oracle (CPU) timing
def time_oracle(model, target_s=15.0, seed=0, k0=4):
    """Times the FP64 oracle's formal solve on a bounded sample of origin points, grown
    until it takes about target_s seconds; returns solves/s, threads and the sample."""
    from oracle import Oracle
    threads = os.cpu_count() or 1
    o = Oracle(model, nthreads=threads)
    pops = o.lte()
    rng = np.random.default_rng(seed)
    P = o.dirs.shape[0] // 2
    F = model.species.n_lines * o.Q
    k = k0
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


# ------------------------------------------------------------------ ALI time to converge
def train_clumpy_network(species, n_models=100, n_points=3000, seed0=1000):
    """Network for learned initial populations of the clumpy cloud's species: converged
    populations of seeded cloud and disc models with that species (seeds from seed0,
    held out from the evaluated model) -> trained in the library's BF16 kernels."""
    from paper_1912_08445_gb300 import learned
    t0 = time.perf_counter()
    models = learned.corpus_models(n_models, seed0, n_points=n_points, species=species)
    X, Y, reps = learned.build_corpus(models, ng_period=4)
    corpus_s = time.perf_counter() - t0
    net, trep = learned.train_network(X, Y, species.n_lev, epochs=30, batch=4096, lr=2e-3)
    return net, {"corpus_models": n_models, "corpus_points_each": n_points, "corpus_rows": int(X.shape[0]),
                 "corpus_seconds": round(corpus_s, 2), "train_seconds": round(trep["seconds"], 2),
                 "loss_first_last": [round(trep["first_loss"], 4), round(trep["last_loss"], 4)]}


def ali_time_to_converge(model, net, stream, tol=1e-6, max_iter=300):
    """ALI from LTE (FP64 and mixed) and from the network (mixed) to a max relative change
    below tol, Ng off and on; the rays are traced beforehand (untimed). The timed region
    covers the initial populations (the network's inference included) and the whole
    iteration loop, with a device synchronisation on both sides."""
    import torch
    import paper_1912_08445_gb300 as mg
    tune = mg.Context(precision=mg.MG_MIXED)
    tune.set_stream(stream.cuda_stream)
    tune.load_model(model)
    tune.trace_rays()
    tune.init_populations()
    variant = tune.autotune(reps=1)[0]
    tune.close()
    runs = {}
    for ng in (0, 4):
        for name, prec, start in (("fp64_lte", mg.MG_FP64, "lte"), ("mixed_lte", mg.MG_MIXED, "lte"),
                                  ("mixed_network", mg.MG_MIXED, "network")):
            ctx = mg.Context(precision=prec, tol=tol, max_iter=max_iter, ng_period=ng)
            ctx.set_stream(stream.cuda_stream)
            ctx.load_model(model)
            ctx.trace_rays()
            if prec == mg.MG_MIXED:
                ctx.set_variant(variant)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if start == "lte":
                ctx.init_populations()
            else:
                ctx.init_populations_mlp(net)
            rep, rc = ctx.iterate(allow_not_converged=True)
            torch.cuda.synchronize()
            runs[f"{name}_ng{ng}"] = {"seconds": round(time.perf_counter() - t0, 5), "iterations": rep["iterations"],
                                      "converged": bool(rep["converged"])}
            ctx.close()
    return runs, variant


def fp64_elimination(stream, variant, n_points=10_000):
    """The disc's construction at n_points: one ALI step in FP32 and one with the cells of
    optical depth above 1e2 (diagonal ALO weight >= 1 - 1/100) solved again in FP64, from
    the same LTE start; the promoted share, both times, and the largest relative
    differences of J and of the populations after the step."""
    import torch
    import paper_1912_08445_gb300 as mg
    import synthetic as syn
    m = syn.model_disc(n=n_points, seed=0, n_h2_in=DISC_N_H2_IN)
    out = {"n_points": n_points, "tau_fp64": DISC_TAU_FP64}
    res = {}
    for tau in (0.0, DISC_TAU_FP64):
        c = mg.Context(precision=mg.MG_MIXED, tau_fp64=tau)
        c.set_stream(stream.cuda_stream)
        c.load_model(m)
        c.trace_rays()
        c.init_populations()
        c.set_variant(variant)
        c.formal_solve()          # warm-up (kernel loading)
        c.init_populations()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c.formal_solve()
        J = c.get_radiation()[0]
        c.update_populations()
        torch.cuda.synchronize()
        res[tau] = (time.perf_counter() - t0, J, c.get_populations(), c.promoted_cells() if tau > 0 else 0)
        c.close()
    (t32, J32, p32, _), (t64, J64, p64, prom) = res[0.0], res[DISC_TAU_FP64]
    rel = lambda a, b: float(np.max(2 * np.abs(a - b) / (np.abs(a) + np.abs(b))))
    out.update(promoted_cells=int(prom), promoted_share=round(prom / n_points, 4), step_s_fp32=round(t32, 4),
               step_s_with_fp64=round(t64, 3), slowdown=round(t64 / t32, 1), J_max_rel_diff=rel(J32, J64),
               populations_max_rel_diff=rel(p32, p64))
    return out


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch
    import torch.distributed as dist
    import paper_1912_08445_gb300 as mg
    import synthetic as syn

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    clumpy_mode = args.workload == "clumpy"
    spec = CLUMPY if clumpy_mode else WORKLOAD
    tau_fp64 = 0.0
    model = build_clumpy(seed=rank) if clumpy_mode else build_model(seed=rank)
    n, lev = model.n, model.species.n_lev
    # launch variant: autotuned on the model itself (clumpy cloud) or on a 20k-point disc
    # of the same construction (a full-size disc trial costs a formal solve per variant)
    small = model if clumpy_mode else syn.model_disc(n=20_000, seed=rank, n_h2_in=DISC_N_H2_IN)
    tune = mg.Context(precision=mg.MG_MIXED)
    tune.set_stream(stream.cuda_stream)
    tune.load_model(small)
    tune.trace_rays()
    tune.init_populations()
    variant, _, n_tried = tune.autotune(reps=2)
    tune.close()

    def make_ctx(profile):
        c = mg.Context(device=local, precision=mg.MG_MIXED, profile=profile, tau_fp64=tau_fp64)
        c.set_stream(stream.cuda_stream)
        c.load_model(model)
        st_, _ = c.trace_rays()
        c.init_populations()
        c.set_variant(variant)
        return c, st_

    ctx, st = make_ctx(0)
    solves, updates = ctx.work_counts()

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
        promoted = ctx.promoted_cells()
        ctx.formal_solve()   # (untimed) radiation field of the final populations
        max_L = float(np.max(ctx.get_radiation()[1]))
        feats = ctx.features()
        ctx.close()

        # per-kernel times and executed work (events on the same stream, profiling context)
        ctx, _ = make_ctx(1)
        step()
        ctx.reset_kernel_times()
        kreps = max(2, min(args.steps, 3))
        for _ in range(kreps):
            step()
        kt = ctx.kernel_times()
        executed = ctx.executed_work() / kreps

        # end to end through the C ABI with pinned host buffers
        e2e_steps = max(2, min(args.steps, 5))
        h_in = torch.empty((n, lev), dtype=torch.float64, pin_memory=True).numpy()
        h_out = torch.empty((n, lev), dtype=torch.float64, pin_memory=True).numpy()
        h_in[:] = ctx.get_populations()
        ctx.set_populations(h_in); step(); ctx.get_populations(out=h_out)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ctx.set_populations(h_in)
            step()
            ctx.get_populations(out=h_out)
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps * args.steps
        ctx.close()

    ms_max, e2e_ms_max = reduce_max([ms, e2e_ms], device=f"cuda:{local}")
    if ws > 1:
        dist.barrier()

    if rank == 0:
        pk, pk_kind = peaks()
        rates = mg.measure_pipe_rates(local)
        k_ms, k_n = kt.get("feautrier_mixed", (float("nan"), 1))
        k_avg = k_ms / max(k_n, 1)
        upd_s = executed / (k_avg * 1e-3)
        fma_peak = max(rates["ffma"], rates["ffma2"])       # flops/s, FMA = 2
        op_peak = fma_peak / 2.0                            # FP32 operations/s on the FMA pipe
        achieved = FMA_OPS_PER_UPDATE * upd_s
        mufu_time = upd_s * (MUFU_PER_UPDATE[0] / rates["ex2"] + MUFU_PER_UPDATE[1] / rates["rcp"])
        hbm_bytes = st["n_elements"] * 16
        traffic = recorded_traffic(variant, "feautrier_warp_clumpy50k.json" if clumpy_mode else
                                   "feautrier_warp_disc200k.json")
        roof = {"bound": "alu", "achieved": round(achieved / 1e12, 3), "peak": round(op_peak / 1e12, 3),
                "unit": "T FP32 ops/s (FMA pipe)", "frac": round(achieved / op_peak, 4), "traffic": traffic,
                "kernel": "k_feautrier_warp (feautrier_mixed)", "kernel_ms": round(k_avg, 3),
                "peak_source": "measured in this run: the FMA pipe's FP32 operation rate, max of scalar FFMA "
                               "and packed FFMA2 (mg_measure_pipe_rates; flops/s / 2)",
                "work": f"{FMA_OPS_PER_UPDATE:g} FP32 operations on the FMA pipe (FMA, MUL, ADD one each) per "
                        "executed point-bin update (counted by the kernel: far-wing points it skips are not work)",
                "flops": {"achieved_tflops": round(FLOPS_PER_UPDATE * upd_s / 1e12, 3),
                          "peak_tflops": round(fma_peak / 1e12, 3),
                          "frac": round(FLOPS_PER_UPDATE * upd_s / fma_peak, 4),
                          "note": f"{FLOPS_PER_UPDATE:g} flops per update with FMA = 2; the MULs and ADDs of the "
                                  "recursion take the FMA pipe like FMAs, so this fraction cannot reach 1"},
                "executed_updates_per_launch": int(executed), "nominal_updates_per_launch": int(updates),
                "mufu_frac": round(mufu_time, 4),
                "mufu_note": "one ex2 and one rcp per update against the measured ex2 and rcp rates",
                "pipe_rates": {k: float(f"{v:.4g}") for k, v in rates.items()},
                "hbm_algorithmic_GBps": round(hbm_bytes / (k_avg * 1e-3) / 1e9, 2),
                "hbm_algorithmic_frac": round(hbm_bytes / (k_avg * 1e-3) / 1e9 / pk["hbm_gbs"], 5),
                "other_kernels_ms": {k: round(v[0] / max(v[1], 1), 3) for k, v in kt.items() if k != "feautrier_mixed"}}
        # the second half of the metric: ALI time to converge on the clumpy cloud
        ali = None
        if args.ali_in_bench and not clumpy_mode:
            clumpy = build_clumpy(seed=0)
            net, train = train_clumpy_network(clumpy.species)
            runs, cvar = ali_time_to_converge(clumpy, net, stream)
            ali = {"metric": "ALI time to converge (max relative population change < 1e-6)", "unit": "s",
                   "higher_is_better": False, "config": dict(CLUMPY, launch_variant=cvar),
                   "runs": runs, "network": train,
                   "speedup_mixed_network_vs_fp64": {
                       f"ng{ng}": round(runs[f"fp64_lte_ng{ng}"]["seconds"] / runs[f"mixed_network_ng{ng}"]["seconds"], 1)
                       for ng in (0, 4)}}
        fp64e = None if (clumpy_mode or not args.fp64e) else fp64_elimination(stream, variant)
        cpu_v, cores, sample = time_oracle(model) if args.cpu_baseline else (None, None, None)
        value = whole_job_rate(solves, args.steps, ws, ms_max)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": dict(spec, precision="mixed (FP32 formal solve, cancellation-free elimination; FP64 "
                           "statistical equilibrium)",
                           l2="inputs larger than L2 (FP32 ray store "
                           f"{st['n_elements'] * 16 / 1e9:.2f} GB read per step)",
                           parallelism=f"replicas x{ws}", solves_per_step=solves,
                           cell_freq_updates_per_step=updates, mean_pair_len=round(st["mean_pair_len"], 1),
                           launch_variant=variant, variants_tried=n_tried, promoted_cells=promoted,
                           max_L=round(max_L, 5), max_tau_sobolev_line0=float(f"{10 ** float(np.max(feats[:, 3])):.3g}"),
                           tau_sobolev_line0_p99=float(f"{10 ** float(np.quantile(feats[:, 3], 0.99)):.3g}")),
            "e2e": {"value": whole_job_rate(solves, args.steps, ws, e2e_ms_max), "unit": UNIT,
                    "h2d_bytes_per_step": n * lev * 8, "d2h_bytes_per_step": n * lev * 8},
            "gpu_launches": 3 * args.steps,
            "clocks": clk,
            "roofline": roof,
            "ali": ali,
            "fp64_elimination": fp64e,
            "cpu_baseline": None if cpu_v is None else {"value": cpu_v, "unit": UNIT, "cores": cores,
                                                        "kind": "oracle", "sample": sample},
            "peaks_source": pk_kind,
        }
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    """The oracle (FP64, all host threads) on the default workload: every step is the
    formal solve of a bounded sample of origin points (16 of the disc's 200k, a few
    seconds), whose rate is the line's value."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    clumpy_mode = args.workload == "clumpy"
    model = build_clumpy(seed=0) if clumpy_mode else build_model(seed=0)
    from oracle import Oracle
    threads = os.cpu_count() or 1
    o = Oracle(model, nthreads=threads)
    pops = o.lte()
    P = o.dirs.shape[0] // 2
    F = model.species.n_lines * o.Q
    k = 256 if clumpy_mode else 16
    rng = np.random.default_rng(0)
    origins = np.sort(rng.choice(model.n, k, replace=False))
    for _ in range(args.warmup):
        o.formal_solve(pops, origins[:2])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        J, L, E = o.formal_solve(pops, origins)
    dt = time.perf_counter() - t0
    solves = k * P * F * args.steps
    v = solves / dt
    spec = CLUMPY if clumpy_mode else WORKLOAD
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(spec, precision="fp64"),
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
    model = build_clumpy(seed=0)
    stream = torch.cuda.Stream()
    out = {"metric": "ALI time to converge (max relative population change < 1e-6)", "unit": "s",
           "higher_is_better": False, "data": "synthetic", "config": dict(CLUMPY), "runs": []}
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
    # the same batched ALI with each model's Ng steps (every 4th iteration)
    ctxs_ng = []
    for m in models:
        c = mg.Context(precision=mg.MG_MIXED, tol=1e-6, max_iter=100, ng_period=4)
        c.load_model(m)
        c.trace_rays()
        c.init_populations()
        ctxs_ng.append(c)
    b_ng = mg.Batch(ctxs_ng)
    b_ng.set_variant(v, srt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps_ng, rc_ng = b_ng.iterate(allow_not_converged=True)
    ali_ng_s = time.perf_counter() - t0
    its_ng = [r["iterations"] for r in reps_ng]
    b_ng.close()
    print(json.dumps({
        "metric": METRIC, "unit": UNIT, "workload": f"{len(models)} clumpy clouds, "
        f"{min(m.n for m in models)}-{max(m.n for m in models)} points, 48 rays, 4 lines x 31 bins",
        "points_total": int(sum(m.n for m in models)), "solves_per_formal_solve": solves,
        "cell_freq_updates": updates, "batched_value": solves / batched, "batched_ms": batched * 1e3,
        "looped_value": solves / looped, "looped_ms": looped * 1e3, "variant": v, "queue_sorted": srt,
        "ali_seconds": ali_s, "ali_iterations_min_max": [min(its), max(its)],
        "ali_converged": int(sum(r["converged"] for r in reps)),
        "ali_ng_seconds": ali_ng_s, "ali_ng_iterations_min_max": [min(its_ng), max(its_ng)],
        "ali_ng_converged": int(sum(r["converged"] for r in reps_ng)), "generation_s": gen_s}))


def run_disc(args):
    """Keplerian disc (200k points, 192 rays, 20-level rotor, 19 lines x 63 bins), mixed
    precision: one ALI iteration per step. With --tau-fp64 T the cells whose diagonal ALO
    weight reaches 1 - 1/T are solved again in FP64 every step."""
    import numpy as np
    import torch
    import paper_1912_08445_gb300 as mg
    import synthetic as syn
    m = syn.model_disc(n=args.disc_points, seed=0, n_h2_in=DISC_N_H2_IN)
    ctx = mg.Context(precision=mg.MG_MIXED, profile=1, tau_fp64=args.tau_fp64)
    ctx.load_model(m)
    t0 = time.perf_counter()
    st, _ = ctx.trace_rays()
    trace_s = time.perf_counter() - t0
    ctx.init_populations()
    if args.variant >= 0:
        v = args.variant
        ctx.set_variant(v)
    else:
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
    ali = None
    if args.disc_ali:   # ALI to 1e-6 from LTE on the same context, Ng every 4th iteration
        ali = {}
        for ng in (4, 0):
            c2 = mg.Context(precision=mg.MG_MIXED, tol=1e-6, max_iter=200, ng_period=ng)
            c2.load_model(m)
            c2.trace_rays()
            c2.set_variant(v)
            c2.init_populations()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            rep, rc = c2.iterate(allow_not_converged=True)
            torch.cuda.synchronize()
            ali[f"mixed_lte_ng{ng}"] = {"seconds": time.perf_counter() - t1, "iterations": rep["iterations"],
                                        "converged": bool(rep["converged"])}
            c2.close()
    print(json.dumps({"metric": METRIC, "unit": UNIT, "ali_to_1e-6": ali, "workload": "Keplerian disc, "
                      f"{m.n} points, 192 rays, 20 levels, 19 lines x 63 bins", "value": solves / dt,
                      "ms_per_step": dt * 1e3, "cell_freq_updates": updates, "variant": v,
                      "tau_fp64": args.tau_fp64, "promoted_cells": ctx.promoted_cells() if args.tau_fp64 > 0 else 0,
                      "max_L": max_L,
                      "trace_s": trace_s, "ray_stats": st, "kernel_ms": {k: v2[0] / max(v2[1], 1) for k, v2 in kt.items()}}))


def run_kernels(args):
    """Every kernel family once on stated cases, for profiling (each launch also timed
    with CUDA events): the ray tracer, line data, warp formal solve and statistical
    equilibrium on the 3D clumpy cloud (50k points, mixed); the FP64 formal solve, the
    band-ALO kernels (bandwidth 1) and the scattering iteration on a 2000-point cloud."""
    import torch
    import paper_1912_08445_gb300 as mg
    import synthetic as syn
    out = {"cases": {}}
    big = build_clumpy(seed=0)
    c = mg.Context(precision=mg.MG_MIXED, profile=1)
    c.load_model(big)
    c.trace_rays()
    c.init_populations()
    if args.variant >= 0:   # the warp kernel's launch variant (else the model's default)
        c.set_variant(args.variant)
    c.formal_solve()
    c.update_populations()
    torch.cuda.synchronize()
    out["cases"]["clumpy50k_mixed"] = {k: round(v[0] / max(v[1], 1), 4) for k, v in c.kernel_times().items()}
    out["cases"]["clumpy50k_mixed"]["executed_updates"] = c.executed_work()
    c.close()
    small = syn.model_clumpy_3d(n=2000, seed=1)
    for name, opts, sca in (("clumpy2k_fp64", {}, False), ("clumpy2k_fp64_band1", {"alo_band": 1}, False),
                            ("clumpy2k_fp64_scattering", {}, True)):
        c = mg.Context(precision=mg.MG_FP64, profile=1, **opts)
        c.load_model(small)
        c.trace_rays()
        c.init_populations()
        if sca:
            c.set_scattering(3e-14 * small.n_coll / small.n_coll.max(), tol=1e-10, max_iter=50)
        c.formal_solve()
        c.update_populations()
        torch.cuda.synchronize()
        rec = {k: round(v[0] / max(v[1], 1), 4) for k, v in c.kernel_times().items()}
        if opts:
            rec["gmres_iterations"] = c.band_status()[1]
        if sca:
            rec["scattering_passes"] = c.scattering_status()[0]
        out["cases"][name] = rec
        c.close()
    print(json.dumps(out))


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
    train = learned.corpus_models(args.corpus, 1000, n_points=args.corpus_points, species=sp,
                                  abundance_range=(1e-7, 1e-4))
    X, Y, reps = learned.build_corpus(train, ng_period=4)
    corpus_s = time.perf_counter() - t0
    net, trep = learned.train_network(X, Y, 20, epochs=args.epochs, batch=4096, lr=2e-3)
    held = learned.corpus_models(10, 5000, n_points=args.corpus_points, species=sp, abundance_range=(1e-7, 1e-4))
    slow = learned.slow_discs((5101, 5102), n_points=args.corpus_points, species=sp)
    for m in slow:
        m.name = "disc_slow"
    rows = []
    for m in held + slow:
        for ng in (0, 4):
            rec = {"n": m.n, "shape": m.name, "ng_period": ng}
            starts, final = {}, None
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
                if prec == mg.MG_MIXED:   # (untimed) the start and the fixed point it reached
                    final = ctx.get_populations()
                    if start == "lte":
                        ctx.init_populations()
                    else:
                        ctx.init_populations_mlp(net)
                    starts[start] = ctx.get_populations()
                ctx.close()
            # distance of each start from the fixed point (levels above 1e-6 of the species)
            big = final >= 1e-6 * final.sum(axis=1, keepdims=True)
            for start, p0 in starts.items():
                rec[f"start_error_{start}"] = float(np.max(np.abs(p0[big] - final[big]) / final[big]))
            rows.append(rec)
    summ = {}
    for ng, group in ((0, "held_out"), (4, "held_out"), (0, "slow_discs"), (4, "slow_discs")):
        sel = [r for r in rows if r["ng_period"] == ng and (r["shape"] == "disc_slow") == (group == "slow_discs")]
        key = "" if group == "held_out" else "slow_"
        for name in ("fp64_lte", "mixed_lte", "mixed_mlp"):
            summ[f"{key}{name}_ng{ng}"] = {"mean_seconds": float(np.mean([r[name]["seconds"] for r in sel])),
                                           "mean_iterations": float(np.mean([r[name]["iterations"] for r in sel])),
                                           "all_converged": all(r[name]["converged"] for r in sel)}
        summ[f"{key}iteration_gain_ng{ng}"] = [round(1 - r["mixed_mlp"]["iterations"] / r["mixed_lte"]["iterations"], 3)
                                               for r in sel]
        # the iterations a start saves if the error falls by a constant factor rho per
        # iteration: log(e_lte / e_mlp) / log(1 / rho), rho from the LTE run to 1e-6
        pred = []
        for r in sel:
            e_l, e_m, it = r["start_error_lte"], r["start_error_mlp"], r["mixed_lte"]["iterations"]
            rho = (1e-6 / e_l) ** (1.0 / it) if e_l > 1e-6 and it > 0 else float("nan")
            pred.append(round(float(np.log(e_l / e_m) / np.log(1.0 / rho)), 2) if 0 < rho < 1 else None)
        summ[f"{key}start_error_lte_ng{ng}"] = [float(f"{r['start_error_lte']:.3g}") for r in sel]
        summ[f"{key}start_error_mlp_ng{ng}"] = [float(f"{r['start_error_mlp']:.3g}") for r in sel]
        summ[f"{key}predicted_iterations_saved_ng{ng}"] = pred
    # the band-diagonal ALO (FP64 contexts) on the slow discs, Ng off: the method's own
    # means of cutting these iterations, beside the network's start
    band_rows = []
    for m in slow:
        rec = {"n": m.n, "shape": m.name}
        for band in (1, 2):
            ctx = mg.Context(precision=mg.MG_FP64, tol=1e-6, max_iter=400, ng_period=0, alo_band=band)
            ctx.load_model(m)
            ctx.trace_rays()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            ctx.init_populations()
            rep, rc = ctx.iterate(allow_not_converged=True)
            torch.cuda.synchronize()
            rec[f"fp64_band{band}"] = {"seconds": time.perf_counter() - t1, "iterations": rep["iterations"],
                                       "converged": bool(rep["converged"]), "band_in_use": rep["alo_band"]}
            ctx.close()
        band_rows.append(rec)
    for band in (1, 2):
        summ[f"slow_fp64_band{band}_ng0"] = {
            "mean_seconds": float(np.mean([r[f"fp64_band{band}"]["seconds"] for r in band_rows])),
            "mean_iterations": float(np.mean([r[f"fp64_band{band}"]["iterations"] for r in band_rows])),
            "all_converged": all(r[f"fp64_band{band}"]["converged"] for r in band_rows),
            "band_in_use": [r[f"fp64_band{band}"]["band_in_use"] for r in band_rows]}
    print(json.dumps({"metric": "ALI time to converge (1e-6), held-out seeds", "unit": "s", "higher_is_better": False,
                      "workload": f"20-level rotor, cloud/disc models of {args.corpus_points} points, 48 rays, 19 lines x 31 bins; "
                                  "held-out seeds, plus slow discs (X = 1e-4, n_H2(r_in) 1e12-1e13 m^-3)",
                      "corpus_models": len(train), "corpus_rows": int(X.shape[0]), "corpus_seconds": corpus_s,
                      "training": trep, "summary": summ, "runs": rows, "band_runs": band_rows}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-ali", dest="ali_in_bench", action="store_false",
                    help="leave out the ALI time-to-converge half of the default line")
    ap.add_argument("--no-fp64e", dest="fp64e", action="store_false",
                    help="leave out the FP64-elimination record of the default line")
    ap.add_argument("--variant", type=int, default=-1,
                    help="disc and kernels workloads: launch variant of the warp kernel (-1: autotune / default)")
    ap.add_argument("--disc-ali", action="store_true", help="disc workload: also the ALI to 1e-6 from LTE")
    ap.add_argument("--ali", action="store_true", help="measure ALI time to converge instead")
    ap.add_argument("--workload", default="default",
                    choices=["default", "clumpy", "batch", "disc", "learned", "image", "sphere1d", "kernels"])
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
    elif args.workload == "kernels":
        run_kernels(args)
    elif args.ali:
        run_ali(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
