"""Benchmark of the adaptive pseudo-spectral BDF2 step for the 2D FCH flow.

Workload: 1024^2 grid, adaptive IMEX-BDF2 with sigma_tol = 1e-5, critical-case
parameters (q = 0, eta1 = 1.45 eps, eta2 = 1.5 eps, d = 0.75), seeded random
bilayer network initial data. Precision (default fp32x2): transforms and pointwise
stages in double-float arithmetic (pairs of floats, FP64-class accuracy on the
FP32 pipe), norms, energy, mass and controller in double; --prec fp64 runs every
stage in double, --prec mixed in single precision.

One step = one trial of the adaptive algorithm (Sec. 3.2): the IMEX-BDF2 trial
(eq. IMEX-eq, 4 real 2D transforms), F of the trial (4 transforms), the AM3
predictor and relative-L2 error, and the accept/reject + next-step decision, all
on the device. L2 is flushed (a 512 MiB write) before every timed step; each
step is timed with CUDA events on the library's stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs an independent replica on its own GPU (the path
has no exchange step); value = steps of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 1024
SIGMA = 1e-5
T_FINAL = 10.0
METRIC = "BDF2 steps/s (adaptive IMEX-BDF2 trial steps at 1024^2)"
PREC_TEXT = {
    "fp32x2": "double-float (FP32-pair) transforms/pointwise, FP64 reductions/controller",
    "fp64": "FP64 transforms/pointwise/reductions/controller",
    "mixed": "FP32 transforms/pointwise, FP64 reductions/controller",
}


def config(prec: str):
    return {"workload": "adaptive IMEX-BDF2, 1024x1024 periodic grid on [-2pi,2pi)^2, "
                        f"{PREC_TEXT[prec]}, sigma_tol=1e-5, critical eta1/eta2 (pearling "
                        "regime), seeded random bilayer network init",
            "n": N_GRID, "scheme": "imex", "precision": prec, "sigma_tol": SIGMA,
            "l2": "flushed before every timed step (512 MiB write)"}


def rank_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def job_throughput(local_ms: float, steps: int, world: int, device=None):
    """Whole-job steps/s of independent replicas: every rank ran `steps` steps in
    local_ms of device time; the job's time is the slowest rank's (max over
    ranks, after a barrier), and value = world * steps / that time."""
    t_ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([t_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
        dist.barrier()
    return world * steps / (t_ms / 1e3), t_ms


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu: int):
        self.gpu, self.proc, self.lines = gpu, None, []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi takes a moment to start: wait for its first sample so that the
            # samples kept (from here on) fall inside the timed region
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        self.start = len(self.lines)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            # one more sample, taken as the region ends, for regions shorter than the period
            n, t0 = len(self.lines), time.time()
            while len(self.lines) == n and len(self.lines) == self.start and time.time() - t0 < 0.3:
                time.sleep(0.01)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[getattr(self, "start", 0):]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def profile_table(name: str):
    """rows of a whitespace table in profiles/<name> (ncu-derived figures)"""
    rows = []
    try:
        for line in open(os.path.join(ROOT, "profiles", name)):
            f = line.split("#")[0].split()
            if f:
                rows.append(f)
    except OSError:
        pass
    return rows


def _profile_value(name: str, prec: str, kernel: str, n: int):
    for r in profile_table(name):
        if len(r) >= 4 and r[0] == prec and r[1] == kernel and int(r[2]) == n:
            return float(r[3])
    return None


def compulsory_bytes(name: str, n: int, csz: int):
    """Compulsory HBM bytes of one launch of a pass (SURVEY 8(d) accounting): the
    arrays of the step's own inputs and outputs it must read or write, once. The
    trial reads u^n, u^{n-1}, F(u^n), F(u^{n-1}) and writes u~, F(u~) (6H in all);
    the work array between the passes and the real-space fields a trial keeps for the
    next one are intermediates (L2-resident) and do not count. H = one half spectrum
    (n/2+1) n complex elements of csz bytes."""
    H = (n // 2 + 1) * n * csz
    table = {
        "row_nimex_direct": 2 * H,     # u^n, u^{n-1} (read in their kept real-space form)
        "row_sav_direct": 2 * H,
        "col_imex_solve": 3 * H,       # u^n, u^{n-1} in; u~ out (eq. IMEX-eq)
        "col_f_finish": 5 * H,         # u~, u^n, F(u^n), F(u^{n-1}) in; F(u~) out (eq. Predictor)
        "row_f": None,                 # intermediates only
    }
    return table.get(name)


def method_flops(name: str, n: int):
    """Floating-point operations the method itself needs in one launch of a pass
    (SURVEY 8(d)): 2.5 n^2 log2(n^2) per 2D real transform, a row or column pass
    doing one half of each transform it touches, plus the pointwise flops of the
    pass per grid point (the IMEX step's ~60 a point split over its passes)."""
    T = 2.5 * n * n * math.log2(n * n)
    table = {
        "row_nimex_direct": T + 40 * n * n,    # W', W'' and N_IMEX pieces; forward rows of 2 fields
        "col_imex_solve": 2 * T + 10 * n * n,  # forward columns of 2, solve, inverse columns of 2
        "row_f": 2 * T + 50 * n * n,           # inverse rows of 2, mu pieces, forward rows of 2
        "col_f_finish": T + 15 * n * n,        # forward columns of 2, F, AM3, two norms
    }
    return table.get(name)


def roofline(prec: str, kernel: str, n: int, launch_ms: float, alu: dict, ms_per_step: float):
    """Roofline of the dominant pass against the measured HBM copy bandwidth:
    achieved = compulsory bytes of one launch (compulsory_bytes) over the live mean
    launch time. Beside it: the same launch's method flops (method_flops) against the
    measured FMA-pipe peak of its precision (the FP32 pipe for double-float and single
    precision, the FP64 pipe for double), the pipe use of the floating-point
    instructions the kernel executes (ncu SASS counts, profiles/flops_per_launch.txt),
    and the whole trial's compulsory bytes (6H) over the time per step."""
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs") or 6800.0
    t = launch_ms / 1e3
    csz = 8 if prec == "mixed" else 16
    cb = compulsory_bytes(kernel, n, csz)
    ach = cb / t / 1e9 if cb else None
    pipe = "fp64" if prec == "fp64" else "fp32"
    peak_flops = alu.get(pipe)
    mf = method_flops(kernel, n)
    sass = _profile_value("flops_per_launch.txt", prec, kernel, n)
    H = (n // 2 + 1) * n * csz
    return {
        "kernel": kernel, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
        "frac": ach / hbm if ach else None,
        "traffic": _profile_value("dram_traffic.txt", prec, kernel, n),
        "compulsory_bytes_per_launch": cb, "avg_launch_us": launch_ms * 1e3,
        "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks.get("hbm_gbs")
        else "fallback 6800 GB/s (of fallback)",
        "method_flops_view": {
            "flops_per_launch": mf, "achieved_tflops": mf / t / 1e12 if mf else None,
            "peak_tflops": peak_flops / 1e12 if peak_flops else None,
            "frac": mf / t / peak_flops if mf and peak_flops else None,
            "peak_source": f"measured {pipe.upper()} FMA pipe (fch_alu_peak, {alu.get('sms')} SMs)"},
        "pipe_use": {
            "sass_flops_per_launch": sass, "achieved_tflops": sass / t / 1e12 if sass else None,
            "frac": sass / t / peak_flops if sass and peak_flops else None,
            "source": "ncu SASS op counts (fadd + fmul + 2 ffma, or the d- forms), "
                      "profiles/flops_per_launch.txt, over the measured pipe peak"},
        "step_view": {"compulsory_bytes_per_step": 6 * H,
                      "achieved_gbs": 6 * H / (ms_per_step / 1e3) / 1e9,
                      "frac": 6 * H / (ms_per_step / 1e3) / 1e9 / hbm},
    }


def run_gb300(args):
    import numpy as np
    import torch

    rank, world, local = rank_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2006_04784_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2006_04784_gb300 import fch
    from paper_2006_04784_gb300 import inputs as I

    n = N_GRID
    prec = {"mixed": fch.FCH_MIXED, "fp64": fch.FCH_FP64, "fp32x2": fch.FCH_FP32X2}[args.prec]
    p = fch.params_default(0.0, eta2=1.5 * 0.1, prec=prec, sync_every=64, autotune=int(args.autotune))
    tiles = ((fch.autotune_step if args.autotune == 2 else fch.autotune)(n, prec)
             if args.autotune else None)
    u0 = I.random_network(n, d=0.75, seed=3 + rank)
    stream = torch.cuda.Stream(device=dev)
    # the arithmetic peaks of this GPU (denominators of the passes' ALU views)
    f32, sms = fch.alu_peak(fch.FCH_MIXED, stream)
    f64, _ = fch.alu_peak(fch.FCH_FP64, stream)
    alu = {"fp32": f32, "fp64": f64, "sms": sms}
    ctx = fch.Context(n, p, stream=stream)
    ctx.set_state(u0)
    ctx.adaptive_begin(args.scheme, SIGMA, T_FINAL)
    ctx.adaptive_enqueue(max(args.warmup, 3))
    ctx.synchronize()
    st0 = ctx.stats()

    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    K = args.steps

    def timed_steps(k):
        """k trial steps, L2 flushed before each, each bracketed by CUDA events on
        the library's stream; returns the per-step device times in ms."""
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(k)]
        with torch.cuda.stream(stream):
            for i in range(k):
                flush.fill_(float(i))
                evs[i][0].record(stream)
                ctx.adaptive_enqueue(1)
                evs[i][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    # region 1 (the metric): trials replay the captured CUDA graph of one trial
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        step_ms = timed_steps(K)
    st1 = ctx.stats()
    # region 2 (per-kernel durations for the roofline): the same trials launched
    # one kernel at a time with events around every launch
    K2 = min(K, 300)
    ctx.pass_timing(True)
    ctx.pass_times()  # clear
    step_ms_eager = timed_steps(K2)
    times = ctx.pass_times()
    ctx.pass_timing(False)
    ctx.adaptive_end()
    value, tot_ms = job_throughput(sum(step_ms), K, world, dev)
    ms_per_step = tot_ms / K
    nfft = st1["n_fft"] - st0["n_fft"]
    eager_ms_per_step = sum(step_ms_eager) / K2
    # dominant kernel and its roofline
    dom = max((k for k in times if k != "ctrl"), key=lambda k: times[k][0])
    dms, dn = times[dom]
    roof = roofline(args.prec, dom, n, dms / dn, alu, ms_per_step)
    kernels = {k: {"ms_total": round(v[0], 4), "launches": v[1],
                   "share": round(v[0] / sum(x[0] for x in times.values()), 4)}
               for k, v in sorted(times.items(), key=lambda kv: -kv[1][0])}

    out = None
    if rank == 0:
        e2e = e2e_measure(fch, I, p, n, dev, min(K, 200))
        out = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": K,
               "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None,
               "dtype": {"fp32x2": "f32x2+f64", "fp64": "f64", "mixed": "f32+f64"}[args.prec],
               "data": "synthetic (seeded random bilayer network, no dataset)",
               "config": dict(config(args.prec), parallelism="replicas" if world > 1 else "single"),
               "ffts_per_s": world * nfft / (tot_ms / 1e3),
               "ffts_per_step": nfft / K,
               "accepted": st1["n_steps"] - st0["n_steps"], "rejected": st1["n_rejects"] - st0["n_rejects"],
               "t_reached": st1["t"],
               "gpu_launches": sum(v[1] for v in times.values()) // max(1, K2) * K,  # per trial, from the eager region
               "tiles": tiles, "kernels": kernels, "kernels_region": f"{K2} trials launched kernel by kernel "
               f"(per-launch events; {eager_ms_per_step:.4f} ms/step there vs {ms_per_step:.4f} "
               "with the CUDA graph)", "roofline": roof, "clocks": clk.summary(), "e2e": e2e,
               "alu_peaks": {"fp32_tflops": f32 / 1e12, "fp64_tflops": f64 / 1e12, "sms": sms,
                             "source": "fch_alu_peak: independent FMA chains, best of 5 launches"}}
        if not args.no_fft:
            out["fft"] = fft_throughput(fch, dev, alu)
            out["fixed_step"] = fixed_step_throughput(fch, I, dev)
        if not args.no_t_final and world == 1:
            out["time_to_t_final"] = time_to_t_final(fch, I, n)
        if not args.no_ensemble and world == 1:
            # the batched ensemble (64 instances on 256^2 to 1024^2 grids, one graph a launch)
            out["ensemble"] = ensemble_bench(args)
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = cpu_baseline(args)
    ctx.close()
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return out


def time_to_t_final(fch, I, n, t_final=0.02):
    """Wall time of fch_run_adaptive from the initial data to t_final at sigma_tol,
    per precision, and the relative L2 error at t_final against a reference run
    (double-float at sigma_tol/100; the global error scales like sigma^(2/3))."""
    import numpy as np

    u0 = I.random_network(n, d=0.75, seed=3)

    def run(prec, sigma, budget=0):
        p = fch.params_default(0.0, eta2=0.15, prec=prec, sync_every=64)
        with fch.Context(n, p) as ctx:
            ctx.set_state(u0)
            t0 = time.perf_counter()
            st = ctx.run_adaptive("imex", sigma, t_final, max_attempts=budget, raise_on_timeout=False)
            wall = time.perf_counter() - t0
            return st, wall, ctx.get_state()

    ref_st, ref_wall, ref = run(fch.FCH_FP32X2, SIGMA / 100)
    out = {"t_final": t_final, "sigma_tol": SIGMA,
           "reference": {"precision": "fp32x2", "sigma_tol": SIGMA / 100, "trials": ref_st["n_attempts"],
                         "wall_s": ref_wall}}
    for name, prec, budget in (("fp32x2", fch.FCH_FP32X2, 0), ("fp64", fch.FCH_FP64, 0),
                               ("mixed", fch.FCH_MIXED, 3000)):
        st, wall, u = run(prec, SIGMA, budget)
        reached = st["t"] >= t_final * (1 - 1e-12)
        out[name] = {"wall_s": wall, "trials": st["n_attempts"], "rejected": st["n_rejects"],
                     "t_reached": st["t"], "reached": bool(reached),
                     "rel_l2_error": float(np.linalg.norm(u - ref) / np.linalg.norm(ref)) if reached else None}
    return out


def fft_throughput(fch, dev, alu, n=N_GRID, batch=32, iters=10, warmup=3):
    """Standalone 2D real transforms at n^2 (fch_fft_r2c then fch_fft_c2r over a
    batch of fields, inputs larger than L2) against cuFFT through torch.fft
    (rfft2 / irfft2 of the same batch), FP64 and FP32, with the tiles fch_autotune
    picks for (n, precision). One transform = one field one way. Roofline per transform: compulsory bytes (read the field or spectrum,
    write the other) against HBM, and 2.5 n^2 log2(n^2) flops against the measured
    FMA-pipe peak of the precision (alu: fch_alu_peak figures)."""
    import torch

    hbm = measured_peaks().get("hbm_gbs") or 6800.0
    out = {"n": n, "batch": batch, "unit": "2D real transforms/s (one field, one way)"}
    for name, prec, rdt in (("fp64", fch.FCH_FP64, torch.float64), ("fp32", fch.FCH_MIXED, torch.float32)):
        stream = torch.cuda.Stream(device=dev)
        x = torch.randn(batch, n, n, dtype=rdt, device=dev)
        X = torch.empty(batch, n // 2 + 1, n, dtype=torch.complex128 if rdt == torch.float64 else torch.complex64,
                        device=dev)
        y = torch.empty_like(x)
        tiles = fch.autotune(n, prec)  # plans take the tuned tiles of (n, precision)
        plan = fch.FFTPlan(n, prec, stream=stream)

        def ours():
            plan.r2c(x, X)
            plan.c2r(X, y)

        def cufft():
            torch.fft.irfft2(torch.fft.rfft2(x), s=(n, n))

        res = {}
        for label, fn in (("fch", ours), ("cufft", cufft)):
            with torch.cuda.stream(stream):
                for _ in range(warmup):
                    fn()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record(stream)
                for _ in range(iters):
                    fn()
                b.record(stream)
            torch.cuda.synchronize()
            res[label] = 2 * batch * iters / (a.elapsed_time(b) / 1e3)
        err = float((y - x).abs().max() / x.abs().max())
        plan.close()
        rs = 8 if rdt == torch.float64 else 4
        byt = n * n * rs + (n // 2 + 1) * n * 2 * rs
        ent = {"fch": res["fch"], "cufft": res["cufft"], "fch_over_cufft": res["fch"] / res["cufft"],
               "tiles": tiles,
               "round_trip_max_rel_err": err, "bytes_per_transform": byt,
               "hbm_frac": res["fch"] * byt / 1e9 / hbm, "hbm_peak_gbs": hbm}
        fl = 2.5 * n * n * math.log2(n * n)
        pk = alu["fp64" if name == "fp64" else "fp32"]
        ent["pipe_frac"] = res["fch"] * fl / pk
        ent["pipe_peak_tflops"] = pk / 1e12
        ent["pipe_peak_source"] = f"measured {name[:4].upper()} FMA pipe (fch_alu_peak)"
        out[name] = ent
        del x, X, y
    return out


def fft_only(args):
    """the `fft` entry of the benchmark line alone (--fft-only): standalone transforms at
    1024^2 with the tiles fch_autotune picks, against cuFFT"""
    import torch

    from paper_2006_04784_gb300 import build as B
    B.build()
    from paper_2006_04784_gb300 import fch

    dev = torch.device("cuda", 0)
    f32, sms = fch.alu_peak(fch.FCH_MIXED)
    f64, _ = fch.alu_peak(fch.FCH_FP64)
    return fft_throughput(fch, dev, {"fp32": f32, "fp64": f64, "sms": sms}, batch=args.fft_batch,
                          iters=args.fft_iters)


def fno_forward_times(args, sizes=(128, 256, 512, 1024), reps=10):
    """the forward pass of the configured network (32 channels, 4 layers, 16 modes, 64
    projection channels; seeded weights) per grid size, batch 1, in each mode: FP32
    weights and full transforms (0), bfloat16 weights (1), bfloat16 weights and
    truncated-DFT spectral convolutions with the x DFT on the tensor cores (2); times
    from CUDA events around `reps` passes after three untimed ones"""
    import torch

    from paper_2006_04784_gb300 import build as B
    B.build()
    from paper_2006_04784_gb300 import fch
    from paper_2006_04784_gb300 import fno_train as T

    dev = torch.device("cuda", 0)
    net = fch.FNO(32, 4, 16, 64)
    net.set_params(T.init_params(net, seed=0))
    out = {"network": "32 channels, 4 layers, 16 modes, 64 projection channels", "unit": "ms per forward pass",
           "modes": {"0": "fp32", "1": "bf16 weights", "2": "bf16 weights, truncated DFTs, tensor cores"}}
    if args.fno_forward_n:
        sizes = (args.fno_forward_n,)
    modes = (args.fno_forward_mode,) if args.fno_forward_mode >= 0 else (0, 1, 2)
    for n in sizes:
        a = torch.randn((1, 2, n, n), device=dev, generator=torch.Generator(device=dev).manual_seed(n))
        y = torch.empty((1, n, n), device=dev)
        row = {}
        for mode in modes:
            net.set_bf16(mode)
            for _ in range(3):
                net.forward(a, y)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            torch.cuda.synchronize()
            ev[0].record()
            for _ in range(reps):
                net.forward(a, y)
            ev[1].record()
            torch.cuda.synchronize()
            row[str(mode)] = ev[0].elapsed_time(ev[1]) / reps
        out[str(n)] = row
    net.set_bf16(0)
    return out


def fixed_step_throughput(fch, I, dev, n=N_GRID, steps=200, dt=1e-6):
    """Fixed-dt IMEX-BDF2 steps at n^2 (fch_run_fixed: a captured step replayed),
    per precision, timed with CUDA events on the context's stream (the step's
    working set, ~50 MB in FP32X2, stays in L2 between steps)."""
    import torch

    u0 = I.random_network(n, d=0.75, seed=3)
    out = {"n": n, "dt": dt, "steps": steps, "scheme": "imex", "unit": "steps/s"}
    for name, prec in (("fp32x2", fch.FCH_FP32X2), ("fp64", fch.FCH_FP64), ("fp32", fch.FCH_MIXED)):
        stream = torch.cuda.Stream(device=dev)
        with fch.Context(n, fch.params_default(0.0, eta2=0.15, prec=prec), stream=stream) as ctx:
            ctx.set_state(u0)
            ctx.run_fixed("imex", dt, 5)
            ctx.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.run_fixed("imex", dt, steps)
            b.record(stream)
            ctx.synchronize()
            out[name] = steps / (a.elapsed_time(b) / 1e3)
    return out


def e2e_measure(fch, I, p, n, dev, K):
    """The same metric through the public C ABI with host arrays: set_state from
    a host array, K adaptive trials by fch_run_adaptive (one call per step, each
    pushes the step's scalars and reads back the control block), get_state to a
    host array at the end. Host copies are inside the timed region."""
    import numpy as np
    import torch

    u0 = np.ascontiguousarray(I.random_network(n, d=0.75, seed=3))
    out = np.empty_like(u0)
    ctx = fch.Context(n, p)
    ctx.set_state(u0)
    ctx.run_adaptive("imex", SIGMA, T_FINAL, max_attempts=4, raise_on_timeout=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.set_state(u0)
    for _ in range(K):
        ctx.run_adaptive("imex", SIGMA, T_FINAL, max_attempts=1, raise_on_timeout=False)
    ctx.get_state_into = None
    res = ctx.get_state()
    t1 = time.perf_counter()
    ctx.close()
    ctrl_bytes = fch.geometry(n)["ctrl_bytes"]
    return {"value": K / (t1 - t0), "unit": "steps/s",
            "h2d_bytes_per_step": (8 * n * n) / K + 2 * ctrl_bytes,
            "d2h_bytes_per_step": (8 * n * n) / K + 2 * ctrl_bytes,
            "note": "public API with host arrays: fch_set_state (host u0), one fch_run_adaptive "
                    "call per step (control block in and out), fch_get_state (host) at the end; "
                    "includes the backward-Euler restart of set_state"}


def _oracle_sample(n: int, trials: int, barrier=None, out=None):
    """A bounded sample of the workload on the oracle: the F history of the
    network initial data, then `trials` adaptive IMEX trials, timed. With a barrier
    (all-cores runs) the timed regions of the workers start together."""
    from oracle import oracle as O
    from paper_2006_04784_gb300 import inputs as I

    u0 = I.random_network(n, d=0.75, seed=3)
    s = O.Stepper(n, 4 * math.pi, O.params(eta2=0.15))
    s.set_history(u0, u0, 1e-6)
    s.adaptive_begin("imex", SIGMA, T_FINAL)
    if barrier is not None:
        barrier.wait()
    t0 = time.perf_counter()
    for _ in range(trials):
        s.adaptive_trial()
    dt = time.perf_counter() - t0
    if out is not None:
        out.put(dt)
    return dt


def cpu_baseline(args, trials: int = 2):
    """The oracle as it stands (FP64 C, one thread per process) on a bounded sample
    of the workload: two adaptive IMEX trials at 1024^2, single-threaded, and the
    same sample on every host core at once (one spawned process per core, timed
    regions started together; value = all trials / the slowest worker's time)."""
    import multiprocessing as mp

    from oracle import oracle as O

    O.build()
    n = N_GRID
    dt1 = _oracle_sample(n, trials)
    one = {"value": trials / dt1, "unit": "steps/s", "cores": 1, "kind": "oracle",
           "sample": f"{trials} adaptive IMEX-BDF2 trials at 1024^2 (FP64 oracle, after its F "
                     f"history was built), {dt1:.1f} s, one thread"}
    cores = os.cpu_count() or 1
    try:
        ctx = mp.get_context("spawn")
        bar, q = ctx.Barrier(cores), ctx.Queue()
        ps = [ctx.Process(target=_oracle_sample, args=(n, trials, bar, q)) for _ in range(cores)]
        for p in ps:
            p.start()
        dts = [q.get(timeout=600) for _ in ps]
        for p in ps:
            p.join()
        allc = {"value": cores * trials / max(dts), "unit": "steps/s", "cores": cores, "kind": "oracle",
                "sample": f"{trials} trials per process on {cores} processes (one per host core), "
                          f"slowest {max(dts):.1f} s"}
    except Exception as ex:  # the single-thread figure stands alone
        allc = {"unavailable": f"{type(ex).__name__}: {ex}"}
    return dict(one, all_cores=allc)


def paper_costs(args):
    """The cost comparison of Sec. 5.2 on the super-critical benchmark (Table
    t:Benchmark: q = 0, eta2 = 3 eps, d = 0.5, N = 256, the paper's initial data),
    integrated to T = 250 by each scheme at the sigma_tol the paper quotes, with the
    number of 2D real transforms and the global relative L2 error at T against a
    reference run (IMEX at sigma_tol = 1e-9). FP32X2 throughout."""
    import numpy as np

    from paper_2006_04784_gb300 import build as B
    B.build()
    from paper_2006_04784_gb300 import fch
    from paper_2006_04784_gb300 import inputs as I

    b = I.BENCHMARKS["supercritical"]
    n, T = b["N"], args.paper_T
    u0 = I.paper_initial_data(n, b["d"])

    def run(scheme, sigma):
        p = fch.params_default(b["q"], eta1=b["eta1"] * 0.1, eta2=b["eta2"] * 0.1,
                               prec=fch.FCH_FP32X2, sync_every=256)
        with fch.Context(n, p) as ctx:
            ctx.set_state(u0)
            t0 = time.perf_counter()
            st = ctx.run_adaptive(scheme, sigma, T)
            wall = time.perf_counter() - t0
            return st, wall, ctx.get_state(), ctx.mass(), ctx.energy()

    ref_st, ref_wall, ref, m_ref, e_ref = run("imex", 1e-9)
    out = {"benchmark": "supercritical", "N": n, "T": T, "precision": "fp32x2",
           "fft_unit": "one 2D real transform of one field (R2C or C2R)",
           "reference": {"scheme": "imex", "sigma_tol": 1e-9, "n_fft": ref_st["n_fft"],
                         "steps": ref_st["n_steps"], "wall_s": ref_wall, "mass": m_ref, "energy": e_ref},
           "runs": []}
    for scheme, sigma, paper in (("imex", 3e-6, "1.5e5 FFT calls (Sec. 5.2)"),
                                 ("sav", 3e-6, "2e5 FFT calls (Sec. 5.2; 2.1e5 in Sec. 1)"),
                                 ("psd", 1e-3, "2e5 FFT calls (Sec. 5.2)"),
                                 ("imex", 1e-5, None), ("imex", 1e-6, None),
                                 ("etd", 1e-5, "2.5e6 FFT calls at error 2.5e-3 (Sec. 1)")):
        st, wall, u, m, e = run(scheme, sigma)
        out["runs"].append({"scheme": scheme, "sigma_tol": sigma, "n_fft": st["n_fft"],
                            "steps": st["n_steps"], "rejects": st["n_rejects"],
                            "psd_iter": st["n_psd_iter"], "wall_s": wall,
                            "global_rel_l2": float(np.linalg.norm(u - ref) / np.linalg.norm(ref)),
                            "mass": m, "energy": e, "paper": paper})
    return out


# final times of Table t:Comp-error; the references of Sec. 5.2 (PSD at sigma_tol =
# 1e-9 for q = 0, PSD at 3e-8 for q = 0.2, IMEX at 3e-9 for q = 0.5)
PAPER_T = {"subcritical": 250.0, "critical": 250.0, "supercritical": 250.0, "foot1": 50.0, "foot2": 50.0}
PAPER_REFERENCE = {"supercritical": ("psd", 1e-9), "foot1": ("psd", 3e-8), "foot2": ("imex", 3e-9)}
SIGMA_SWEEP = [1e-3, 3e-4, 1e-4, 3e-5, 1e-5, 3e-6, 1e-6, 3e-7, 1e-7]


PSD_MAX_ITER = [1000]  # PSD iterations per step before FCH_ENOCONV (--psd-max-iter)


def _progress(*a):
    print(*a, file=sys.stderr, flush=True)


def _paper_problem(name):
    """(N, params, initial data) of one benchmark of Table t:Benchmark (eta in units
    of eps = 0.1), FP32X2, default pass tiles (tuned tiles are chosen by timing and
    round differently, which moves the PSD iteration counts from run to run)."""
    from paper_2006_04784_gb300 import fch
    from paper_2006_04784_gb300 import inputs as I

    b = I.BENCHMARKS[name]
    p = fch.params_default(b["q"], eta1=b["eta1"] * 0.1, eta2=b["eta2"] * 0.1,
                           prec=fch.FCH_FP32X2, sync_every=256, psd_max_iter=PSD_MAX_ITER[0])
    return b["N"], p, I.paper_initial_data(b["N"], b["d"])


def _paper_solo(name, scheme, sigma, T, max_attempts=2_000_000):
    """one adaptive run of a benchmark: (stats, wall seconds, final u); a run that
    stops with an error (e.g. PSD's FCH_ENOCONV) returns its stats at that point with
    the error under "error", and u None"""
    from paper_2006_04784_gb300 import fch

    n, p, u0 = _paper_problem(name)
    with fch.Context(n, p) as ctx:
        ctx.set_state(u0)
        t0 = time.perf_counter()
        try:
            st = ctx.run_adaptive(scheme, sigma, T, max_attempts=max_attempts, raise_on_timeout=False)
        except fch.FchError as e:
            st = dict(ctx.stats(), error=str(e))
            _progress(name, scheme, sigma, "stopped:", st)
            return st, time.perf_counter() - t0, None
        wall = time.perf_counter() - t0
        _progress(name, scheme, sigma, f"{wall:.1f} s", st)
        return st, wall, (ctx.get_state() if st["t"] >= T * (1 - 1e-12) else None)


def _paper_ensemble(members, T, rounds=16):
    """members: (benchmark, scheme, sigma) runs of non-PSD schemes, all to the same
    T, advanced together as one ensemble. Returns ([(stats, final u)], wall seconds)."""
    from paper_2006_04784_gb300 import fch

    probs = [_paper_problem(b) for b, _, _ in members]
    with fch.Ensemble([pr[0] for pr in probs], [pr[1] for pr in probs]) as ens:
        for i, pr in enumerate(probs):
            ens[i].set_state(pr[2])
        t0 = time.perf_counter()
        st = ens.run_adaptive_each([m[1] for m in members], [m[2] for m in members], T, rounds=rounds)
        wall = time.perf_counter() - t0
        _progress(f"ensemble of {len(members)} to T = {T}: {wall:.1f} s")
        return [(st[i], ens[i].get_state()) for i in range(len(members))], wall


def _periodic_labels(mask):
    """connected components (4-neighbour) of a boolean field on the periodic grid"""
    import numpy as np
    from scipy import ndimage

    lab, m = ndimage.label(mask)
    parent = list(range(m + 1))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for a, b in ((lab[:, 0], lab[:, -1]), (lab[0, :], lab[-1, :])):
        for x, y in zip(a, b):
            if x and y:
                rx, ry = find(int(x)), find(int(y))
                if rx != ry:
                    parent[rx] = ry
    return len({find(i) for i in range(1, m + 1)})


def _topology(u, level=-0.12):
    """(components, holes) of the bilayer region {u > level} (the contour level of
    Fig. f:contour): a closed bilayer loop is one component with one hole, an open
    (end-capped) curve or a pearl one without; holes = components of the rest - 1"""
    above = u > level
    return _periodic_labels(above), max(0, _periodic_labels(~above) - 1)


def comp_error(args):
    """Table t:Comp-error: relative L2 differences at the final time T between the
    schemes' solutions of each benchmark at sigma_tol = 1e-5 (Sec. 4), FP32X2. The
    IMEX, SAV and ETD runs of all benchmarks with the same T form one ensemble; the
    PSD runs are solo."""
    import numpy as np

    from paper_2006_04784_gb300 import build as B
    B.build()
    sigma = 1e-5
    paper = {"subcritical": (7.276e-3, 7.315e-3, 4.103e-5, None),
             "critical": (2.204e-3, 2.212e-3, 1.796e-5, None),
             "supercritical": (8.817e-2, 8.819e-2, 4.156e-5, 1.568e-2),
             "foot1": (2.358e-3, 2.359e-3, 1.702e-6, None),
             "foot2": (3.318e-4, 3.322e-4, 6.195e-7, None)}
    names = list(paper)
    sols, runs = {}, []
    for T in sorted(set(PAPER_T.values())):
        members = [(b, s, sigma) for b in names if PAPER_T[b] == T
                   for s in (("imex", "sav", "etd") if b == "supercritical" else ("imex", "sav"))]
        res, wall = _paper_ensemble(members, T)
        for (b, s, _), (st, u) in zip(members, res):
            sols[b, s] = u
            runs.append({"benchmark": b, "scheme": s, "T": T, "steps": st["n_steps"], "n_fft": st["n_fft"],
                         "rejects": st["n_rejects"], "t": st["t"]})
        runs.append({"ensemble_T": T, "members": len(members), "wall_s": wall})
    for b in names:
        st, wall, u = _paper_solo(b, "psd", sigma, PAPER_T[b])
        sols[b, "psd"] = u
        runs.append({"benchmark": b, "scheme": "psd", "T": PAPER_T[b], "steps": st["n_steps"],
                     "n_fft": st["n_fft"], "psd_iter": st["n_psd_iter"], "rejects": st["n_rejects"],
                     "t": st["t"], "wall_s": wall, "error": st.get("error")})

    def cell(a, b_):
        return None if a is None or b_ is None else _rel(a, b_)

    # E1: the morphology at T of every run (the paper's descriptions: sub-critical and
    # critical a single closed curve; Foot 1 six closed loops; Foot 2 four loops and
    # two double loops)
    topo = {f"{b}/{sc}": (None if u is None else
                          dict(zip(("components", "holes"), _topology(u))) | {"max_u": float(u.max())})
            for (b, sc), u in sols.items()}

    table = []
    for b in names:
        row = {"benchmark": b, "T": PAPER_T[b],
               "imex/psd": cell(sols[b, "imex"], sols[b, "psd"]),
               "sav/psd": cell(sols[b, "sav"], sols[b, "psd"]),
               "sav/imex": cell(sols[b, "sav"], sols[b, "imex"]),
               "paper": dict(zip(("imex/psd", "sav/psd", "sav/imex", "etd/psd"), paper[b]))}
        if (b, "etd") in sols:
            row["etd/psd"] = cell(sols[b, "etd"], sols[b, "psd"])
        table.append(row)
    return {"table": "t:Comp-error", "sigma_tol": sigma, "precision": "fp32x2",
            "norm": "||u_a - u_b||_2 / ||u_b||_2 over the grid at T", "rows": table, "runs": runs,
            "morphology_at_T": topo}


def _loglog_at(xs, ys, x0):
    """log-log interpolation of y at x = x0 between the first bracketing pair of
    (xs, ys) (xs in sweep order); None when x0 is not bracketed"""
    for i in range(len(xs) - 1):
        a, b = xs[i], xs[i + 1]
        if min(a, b) <= x0 <= max(a, b) and a != b:
            w = (math.log(x0) - math.log(a)) / (math.log(b) - math.log(a))
            return math.exp(math.log(ys[i]) + w * (math.log(ys[i + 1]) - math.log(ys[i])))
    return None


def _slope(xs, ys):
    import numpy as np
    if len(xs) < 2:
        return None
    return float(np.polyfit(np.log(xs), np.log(ys), 1)[0])


def dollars_per_digit(args):
    """Sec. 5.2, Figs. f:BM3-L2 and f:BM4-L2: for one benchmark, the global relative L2
    error at T against a highly accurate run, and the cost in 2D real transforms, as
    sigma_tol sweeps; the cost at the paper's acceptable global error 2.5e-3. IMEX,
    SAV (and ETD on the super-critical benchmark) sweep as one ensemble; PSD runs solo.
    FP32X2."""
    from paper_2006_04784_gb300 import build as B
    B.build()
    name = args.dpd_benchmark
    T = PAPER_T[name]
    ref_scheme, ref_sigma = PAPER_REFERENCE[name]
    ref_st, ref_wall, ref = _paper_solo(name, ref_scheme, ref_sigma, T)
    if ref is None:
        raise RuntimeError(f"reference run failed: {ref_st['error']} at t = {ref_st['t']}")
    sig = [float(x) for x in args.dpd_sigmas.split(",")] if args.dpd_sigmas else SIGMA_SWEEP
    etd_sig = [x for x in sig if x >= args.dpd_etd_min]
    members = [(name, s, x) for s in ("imex", "sav") for x in sig]
    if name == "supercritical":
        members += [(name, "etd", x) for x in etd_sig]
    res, ens_wall = _paper_ensemble(members, T)
    runs = []
    for (_, s, x), (st, u) in zip(members, res):
        runs.append({"scheme": s, "sigma_tol": x, "n_fft": st["n_fft"], "steps": st["n_steps"],
                     "rejects": st["n_rejects"], "t": st["t"], "global_rel_l2": _rel(u, ref)})
    psd_sig = [x for x in sig if x >= args.dpd_psd_min]
    for x in psd_sig:
        st, wall, u = _paper_solo(name, "psd", x, T)
        runs.append({"scheme": "psd", "sigma_tol": x, "n_fft": st["n_fft"], "steps": st["n_steps"],
                     "psd_iter": st["n_psd_iter"], "rejects": st["n_rejects"], "t": st["t"],
                     "wall_s": wall, "global_rel_l2": None if u is None else _rel(u, ref),
                     "error": st.get("error")})
    summary = {}
    for s in ("imex", "sav", "etd", "psd"):
        rs = [r for r in runs if r["scheme"] == s and r["t"] >= T * (1 - 1e-12) and r["global_rel_l2"]]
        if not rs:
            continue
        xs = [r["sigma_tol"] for r in rs]
        err = [r["global_rel_l2"] for r in rs]
        cost = [r["n_fft"] for r in rs]
        fine = [(x, e) for x, e in zip(xs, err) if x <= 1e-5]
        summary[s] = {"n_fft_at_error_2.5e-3": _loglog_at(err, cost, 2.5e-3),
                      "sigma_tol_at_error_2.5e-3": _loglog_at(err, xs, 2.5e-3),
                      "n_fft_at_error_7e-4": _loglog_at(err, cost, 7e-4),
                      "slope_error_vs_sigma(sigma<=1e-5)": _slope([f[0] for f in fine], [f[1] for f in fine]),
                      "slope_n_fft_vs_sigma": _slope(xs, cost)}
    both = [(a["n_fft"], b["n_fft"]) for a in runs if a["scheme"] == "sav"
            for b in runs if b["scheme"] == "imex" and b["sigma_tol"] == a["sigma_tol"]]
    if both:
        summary["sav/imex_n_fft"] = sorted(a / b for a, b in both)[len(both) // 2]
    return {"figure": "f:BM3-L2" if name == "supercritical" else "f:BM4-L2", "benchmark": name, "T": T,
            "N": _paper_problem(name)[0], "precision": "fp32x2",
            "fft_unit": "one 2D real transform of one field (R2C or C2R)",
            "reference": {"scheme": ref_scheme, "sigma_tol": ref_sigma, "n_fft": ref_st["n_fft"],
                          "steps": ref_st["n_steps"], "t": ref_st["t"], "wall_s": ref_wall},
            "ensemble": {"members": len(members), "wall_s": ens_wall},
            "runs": runs, "summary": summary}


TRACE_TIMES = [1, 2, 5, 10, 20, 30, 50, 75, 100, 125, 150, 175, 185, 200, 210, 225, 250]


def traces(args):
    """Time traces on one benchmark (Secs. 4-5): the global relative L2 error against
    the highly accurate run (Fig. f:L2temp_error), the adaptive step size (Fig.
    f:Stepsize) and u - b_- at the domain centre and corner (Fig. f:corner-1), at
    output times up to T, for IMEX, SAV and PSD at sigma_tol = 1e-5, 1e-6, 1e-7 (and
    ETD at 1e-5). Every run advances from output time to output time (the adaptive
    step is clipped at each, reading R4); IMEX, SAV and ETD as one ensemble. FP32X2."""
    from paper_2006_04784_gb300 import build as B
    B.build()
    from paper_2006_04784_gb300 import fch

    name = args.trace_benchmark
    T = PAPER_T[name]
    times = [t for t in TRACE_TIMES if t < T] + [T]
    n, p, u0 = _paper_problem(name)
    ref_scheme, ref_sigma = PAPER_REFERENCE.get(name, ("psd", 1e-9))

    def probe(u):
        c = n // 2  # x = 0 on the grid x0 + i L / n, x0 = -L / 2; the corner is i = 0
        return float(u[c, c] - p.b_minus), float(u[0, 0] - p.b_minus)

    def solo(scheme, sigma):
        rows, states = [], []
        with fch.Context(n, p) as ctx:
            ctx.set_state(u0)
            t0 = time.perf_counter()
            for t in times:
                st = ctx.run_adaptive(scheme, sigma, t, max_attempts=4_000_000, raise_on_timeout=False)
                u = ctx.get_state()
                states.append(u)
                rows.append({"t": st["t"], "k": st["k_last"], "steps": st["n_steps"], "n_fft": st["n_fft"],
                             "centre_corner": probe(u)})
            _progress(name, scheme, sigma, f"{time.perf_counter() - t0:.1f} s")
        return rows, states

    ref_rows, ref_states = solo(ref_scheme, ref_sigma)
    runs = {f"{ref_scheme}_{ref_sigma:g}_reference": ref_rows}
    members = [(s, x) for s in ("imex", "sav") for x in (1e-5, 1e-6, 1e-7)] + [("etd", 1e-5)]
    with fch.Ensemble([n] * len(members), [p] * len(members)) as ens:
        for i in range(len(members)):
            ens[i].set_state(u0)
        rows = [[] for _ in members]
        t0 = time.perf_counter()
        for j, t in enumerate(times):
            st = ens.run_adaptive_each([m[0] for m in members], [m[1] for m in members], t, rounds=16)
            for i in range(len(members)):
                u = ens[i].get_state()
                rows[i].append({"t": st[i]["t"], "k": st[i]["k_last"], "steps": st[i]["n_steps"],
                                "n_fft": st[i]["n_fft"], "centre_corner": probe(u),
                                "global_rel_l2": _rel(u, ref_states[j])})
        _progress(f"ensemble of {len(members)}: {time.perf_counter() - t0:.1f} s")
    for (s, x), r in zip(members, rows):
        runs[f"{s}_{x:g}"] = r
    for x in (1e-5, 1e-6, 1e-7):
        r, states = solo("psd", x)
        for row, u, ur in zip(r, states, ref_states):
            row["global_rel_l2"] = _rel(u, ur)
        runs[f"psd_{x:g}"] = r
    # the mean accepted step over each output interval (the last step before an output
    # time is clipped to it, so k_last there understates the controller's step)
    for r in runs.values():
        for j, row in enumerate(r):
            t_prev, s_prev = (0.0, 0) if j == 0 else (r[j - 1]["t"], r[j - 1]["steps"])
            row["mean_k"] = (row["t"] - t_prev) / max(1, row["steps"] - s_prev)
    return {"figures": ["f:L2temp_error", "f:Stepsize", "f:corner-1"], "benchmark": name, "N": n, "T": T,
            "precision": "fp32x2", "times": times,
            "reference": {"scheme": ref_scheme, "sigma_tol": ref_sigma},
            "probes": "u - b_- at the centre (x = y = 0) and the corner (x = y = -L/2) of the domain",
            "runs": runs}


def _rel(a, b):
    import numpy as np
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cfg1_cpu_baseline(n, u0, p):
    """CPU baseline of the 128^2 fixed-step run: the oracle (single-threaded FP64 C)
    takes the same 400 IMEX steps; returns its timing and final state."""
    from oracle import oracle as O

    O.build()
    s = O.Stepper(n, 4 * math.pi, O.params(eps=p.eps, q=p.q, gamma=p.gamma, eta1=p.eta1, eta2=p.eta2,
                                            zeta=p.zeta, D0=p.D0))
    s.set_state(u0)
    t0 = time.perf_counter()
    for _ in range(400):
        s.step("imex", 1e-3)
    wall = time.perf_counter() - t0
    return {"kind": "oracle", "wall_s": wall, "steps_per_s": 400 / wall, "cores": 1,
            "sample": "the full 400 steps"}, s.state()


def workloads(args):
    """The other configurations of the hot path, measured end to end through the C ABI
    (wall time of the calls, device work included):
    (1) 128^2 circle bilayer, IMEX-BDF2, fixed dt = 1e-3, 400 steps (FP64 and FP32X2),
        with the FP64 result against the oracle's;
    (2) 512^2 multimode bilayer, adaptive IMEX / SAV / PSD / ETD, sigma_tol = 1e-5 to
        t = 50, FP64 and FP32X2: steps, rejects, transforms, PSD iterations, wall time,
        and the FP32X2 - FP64 difference at t = 50;
    (3) 1024^2 and 2048^2 random bilayer network, critical parameters, adaptive IMEX at
        sigma_tol = 1e-5 to t_final: FP32X2 and FP64 wall time and relative L2 error
        against an FP32X2 run at sigma_tol / 100 (FP32 with a trial budget: its LTE
        estimate is rounding-limited at these sizes)."""
    import numpy as np

    from paper_2006_04784_gb300 import build as B
    B.build()
    from paper_2006_04784_gb300 import fch
    from paper_2006_04784_gb300 import inputs as I

    def P(q=0.0, **kw):
        # pass tiles timed on adaptive trials of each grid size and precision
        return fch.params_default(q, **dict({"autotune": 2}, **kw))

    out = {}
    # (1) fixed steps
    n = 128
    u0 = I.circle_bilayer(n)
    cfg1 = {"n": n, "dt": 1e-3, "steps": 400}
    for name, prec in (("fp64", fch.FCH_FP64), ("fp32x2", fch.FCH_FP32X2)):
        with fch.Context(n, P(prec=prec)) as ctx:
            ctx.set_state(u0)
            ctx.synchronize()
            t0 = time.perf_counter()
            for _ in range(400):
                ctx.step("imex", 1e-3)
            ctx.synchronize()
            wall = time.perf_counter() - t0
            u_calls = ctx.get_state()
            ctx.set_state(u0)
            ctx.synchronize()
            t0 = time.perf_counter()
            ctx.run_fixed("imex", 1e-3, 400)
            ctx.synchronize()
            wall_g = time.perf_counter() - t0
            cfg1[name] = {"wall_s": wall_g, "steps_per_s": 400 / wall_g,
                          "steps_per_s_one_call_per_step": 400 / wall, "u": ctx.get_state(),
                          "graph_equals_calls": bool(np.array_equal(ctx.get_state(), u_calls))}
    try:
        cfg1["cpu_baseline"], u_ref = cfg1_cpu_baseline(n, u0, P())
        for name in ("fp64", "fp32x2"):
            cfg1[name]["rel_l2_vs_cpu_baseline"] = _rel(cfg1[name]["u"], u_ref)
    except Exception as e:  # a baseline only
        cfg1["cpu_baseline"] = {"error": str(e)}
    for name in ("fp64", "fp32x2"):
        cfg1[name].pop("u")
    out["cfg1_128_fixed_dt"] = cfg1

    # (2) all schemes at 512^2
    n, T = 512, args.workload_t2
    u0 = I.multimode_bilayer(n)
    cfg2 = {"n": n, "sigma_tol": SIGMA, "t_final": T, "runs": []}
    for scheme in ("imex", "sav", "psd", "etd"):
        res = {}
        for name, prec in (("fp64", fch.FCH_FP64), ("fp32x2", fch.FCH_FP32X2)):
            with fch.Context(n, P(prec=prec, sync_every=256)) as ctx:
                ctx.set_state(u0)
                t0 = time.perf_counter()
                st = ctx.run_adaptive(scheme, SIGMA, T, max_attempts=args.workload_budget,
                                      raise_on_timeout=False)
                wall = time.perf_counter() - t0
                res[name] = {"wall_s": wall, "t_reached": st["t"], "steps": st["n_steps"],
                             "rejects": st["n_rejects"], "transforms": st["n_fft"],
                             "psd_iter": st["n_psd_iter"], "mass": ctx.mass(), "energy": ctx.energy(),
                             "u": ctx.get_state()}
        d = _rel(res["fp32x2"]["u"], res["fp64"]["u"]) if res["fp32x2"]["t_reached"] == res["fp64"]["t_reached"] else None
        for r in res.values():
            r.pop("u")
        cfg2["runs"].append({"scheme": scheme, **res, "fp32x2_vs_fp64_rel_l2": d})
    out["cfg2_512_all_schemes"] = cfg2

    # (3) large grids, adaptive IMEX to t_final
    cfg3 = {"sigma_tol": SIGMA, "t_final": args.workload_t3, "runs": []}
    for n in (1024, 2048):
        u0 = I.random_network(n, d=0.75, seed=3)

        def run(prec, sigma, budget):
            with fch.Context(n, P(eta2=0.15, prec=prec, sync_every=256)) as ctx:
                ctx.set_state(u0)
                t0 = time.perf_counter()
                st = ctx.run_adaptive("imex", sigma, args.workload_t3, max_attempts=budget, raise_on_timeout=False)
                return st, time.perf_counter() - t0, ctx.get_state(), ctx.mass()

        ref_st, ref_wall, ref, _ = run(fch.FCH_FP32X2, SIGMA / 100, 0)
        row = {"n": n, "reference": {"precision": "fp32x2", "sigma_tol": SIGMA / 100,
                                     "steps": ref_st["n_steps"], "wall_s": ref_wall}}
        for name, prec, budget in (("fp32x2", fch.FCH_FP32X2, 0), ("fp64", fch.FCH_FP64, 0),
                                   ("fp32", fch.FCH_MIXED, 2000)):
            st, wall, u, m = run(prec, SIGMA, budget)
            reached = st["t"] >= args.workload_t3 * (1 - 1e-12)
            row[name] = {"wall_s": wall, "t_reached": st["t"], "steps": st["n_steps"], "rejects": st["n_rejects"],
                         "transforms": st["n_fft"], "mass": m,
                         "rel_l2_vs_reference": _rel(u, ref) if reached else None}
        cfg3["runs"].append(row)
    out["cfg3_large_adaptive"] = cfg3
    return out


def ensemble_bench(args):
    """A batched ensemble: 64 instances on uneven grids (32 at 256^2, 24 at 512^2,
    8 at 1024^2), eta1/eps swept linearly over [1, 3], seeds 100..163, multimode
    bilayer initial data, adaptive IMEX-BDF2 at sigma_tol = 1e-5 to t_final, in
    one CUDA graph per launch (fch_ensemble_run_adaptive), against the same 64
    instances run one after another (fch_run_adaptive each). Pass tiles from the
    step tuner (fch_autotune_step) for both unless --ensemble-autotune says otherwise."""
    import numpy as np

    from paper_2006_04784_gb300 import build as B
    B.build()
    from paper_2006_04784_gb300 import fch
    from paper_2006_04784_gb300 import inputs as I

    prec = {"mixed": fch.FCH_MIXED, "fp64": fch.FCH_FP64, "fp32x2": fch.FCH_FP32X2}[args.prec]
    sizes = [256] * 32 + [512] * 24 + [1024] * 8
    m = len(sizes)
    eps = 0.1
    params = [fch.params_default(0.0, eta1=eps * (1.0 + 2.0 * i / (m - 1)), prec=prec, autotune=args.ensemble_autotune,
                                 sync_every=64) for i in range(m)]
    inits = [I.multimode_bilayer(n, seed=100 + i) for i, n in enumerate(sizes)]
    tf = args.ensemble_t
    out = {"members": m, "sizes": {"256": 32, "512": 24, "1024": 8}, "eta1_over_eps": [1.0, 3.0],
           "seeds": [100, 100 + m - 1], "scheme": "imex", "sigma_tol": SIGMA, "t_final": tf,
           "precision": args.prec, "rounds_per_launch": args.ensemble_rounds}
    with fch.Ensemble(sizes, params) as ens:
        for i in range(m):
            ens[i].set_state(inits[i])
        t0 = time.perf_counter()
        st = ens.run_adaptive("imex", SIGMA, tf, rounds=args.ensemble_rounds)
        wall = time.perf_counter() - t0
        ens_states = [ens[i].get_state() for i in (0, 32, 56)]
    trials = sum(s["n_attempts"] for s in st)
    out["ensemble"] = {"wall_s": wall, "trials": trials, "trials_per_s": trials / wall,
                       "steps": sum(s["n_steps"] for s in st), "rejects": sum(s["n_rejects"] for s in st),
                       "all_reached": all(s["t"] >= tf * (1 - 1e-12) for s in st)}
    wall_seq, trials_seq, same = 0.0, 0, True
    for i in range(m):
        with fch.Context(sizes[i], params[i]) as ctx:
            ctx.set_state(inits[i])
            t0 = time.perf_counter()
            s = ctx.run_adaptive("imex", SIGMA, tf)
            wall_seq += time.perf_counter() - t0
            trials_seq += s["n_attempts"]
            if i in (0, 32, 56):
                same = same and bool(np.array_equal(ctx.get_state(), ens_states[(0, 32, 56).index(i)]))
    out["sequential"] = {"wall_s": wall_seq, "trials": trials_seq, "trials_per_s": trials_seq / wall_seq}
    out["speedup"] = wall_seq / wall
    out["members_identical_to_solo_runs"] = same
    return out


def fno_bench(args):
    """The learned PSD initial iterate: a 4-layer FNO (32 channels, 16 modes) trained
    on PSD-BDF2 trajectories the library computes at 128^2 (the 128^2 circle-bilayer
    physics, step sizes 1e-3 x 2^U(-1,1)), then PSD steps started from u* (the plain
    method) and from the FNO's v_0 on held-out trajectories at 128^2 and at 1024^2:
    PSD iterations, initial-iterate error, and the network's inference time."""
    import numpy as np
    import torch

    from paper_2006_04784_gb300 import build as B
    B.build()
    from paper_2006_04784_gb300 import fch
    from paper_2006_04784_gb300 import fno_train as T
    from paper_2006_04784_gb300 import inputs as I

    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(11)
    p = fch.params_default(0.0, psd_itol=1e-10)
    n = 128
    data, t0 = [], time.perf_counter()
    inits = [I.circle_bilayer(n, radius=r, noise=1e-3, seed=s) for r, s in ((1.6, 1), (2.0, 2), (2.4, 3), (1.8, 4))]
    inits += [I.multimode_bilayer(n, r0=r, seed=s) for r, s in ((2.2, 5), (2.8, 6), (3.2, 7), (2.5, 8))]
    for u0 in inits:
        dts = T.random_steps(rng, args.fno_steps, 1e-3)
        data += T.samples_from(T.psd_trajectory(n, u0, dts, p), dts)
    t_data = time.perf_counter() - t0
    net = fch.FNO(32, 4, 16, 64)
    net.set_params(T.init_params(net, seed=0))
    t0 = time.perf_counter()
    hist = T.train(net, data, args.fno_iters, 8, args.fno_lr, dev)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    out = {"network": {"width": 32, "layers": 4, "modes": 16, "proj": 64, "params": net.num_params,
                       "precision": "fp32"},
           "training": {"grid": n, "samples": len(data), "data_s": t_data, "iterations": args.fno_iters,
                        "batch": 8, "lr": args.fno_lr, "train_s": t_train, "loss_first": hist[0],
                        "loss_last10": float(np.mean(hist[-10:]))}}

    def evaluate(m, u0, steps):
        dts = T.random_steps(np.random.default_rng(99), steps, 1e-3)
        it_plain, it_fno, e_plain, e_fno = [], [], [], []
        diffs = []
        # IMEX / SAV with the learned extrapolation: distance of the step to the
        # fully implicit BDF2 step (the PSD fixed point) from u* and from v_0
        gap = {(sc, w): [] for sc in ("imex", "sav") for w in ("plain", "learned")}
        v0 = torch.empty((m, m), dtype=torch.float64, device=dev)
        with fch.Context(m, p) as a, fch.Context(m, p) as b:
            a.set_state(u0)
            hist_u = [np.array(u0)]
            for i, dt in enumerate(dts):
                if i < 2:
                    a.step("psd", dt)
                    hist_u.append(a.get_state())
                    continue
                g = dt / dts[i - 1]
                un, um = hist_u[-1], hist_u[-2]
                ustar = un + g * (un - um)  # for the error figures only
                b.set_history(un, um, dts[i - 1])
                T.learned_start(b, net, v0, dt)  # v_0 on the device from b's history
                b.synchronize()
                a.step("psd", dt)
                it_plain.append(a.stats()["last_psd_iter"])
                # the same BDF2 step (same history) from the learned start
                b.set_history(un, um, dts[i - 1])
                b.step_psd_from(dt, v0)
                it_fno.append(b.stats()["last_psd_iter"])
                u1 = a.get_state()
                diffs.append(float(np.linalg.norm(b.get_state() - u1) / np.linalg.norm(u1)))
                e_plain.append(float(np.linalg.norm(ustar - u1)))
                e_fno.append(float(np.linalg.norm(v0.cpu().numpy() - u1)))
                for sc in ("imex", "sav"):
                    for w in ("plain", "learned"):
                        b.set_history(un, um, dts[i - 1])
                        if w == "plain":
                            b.step(sc, dt)
                        else:
                            b.step_from(sc, dt, v0)
                        gap[sc, w].append(_rel(b.get_state(), u1))
                hist_u.append(u1)
            diff = max(diffs)
        return {"grid": m, "steps": len(it_plain), "psd_iter_plain": float(np.mean(it_plain)),
                "psd_iter_fno": float(np.mean(it_fno)),
                "start_error_ratio": float(np.mean(np.array(e_fno) / np.array(e_plain))),
                "max_rel_diff_learned_vs_plain": diff,
                "learned_extrapolation": {
                    f"{sc}_gap_to_implicit_{w}": float(np.mean(gap[sc, w]))
                    for sc in ("imex", "sav") for w in ("plain", "learned")}}

    out["eval_128"] = evaluate(128, I.circle_bilayer(128, radius=2.1, noise=1e-3, seed=21), 30)
    out["eval_1024"] = evaluate(1024, I.circle_bilayer(1024, radius=2.1, noise=1e-3, seed=21), 8)

    # the adaptive PSD run (sigma_tol = 1e-6) at 1024^2, trial by trial, from u* and from v_0
    ad = {"grid": 1024, "sigma_tol": 1e-6, "t_final": args.fno_t_adaptive}
    u0 = I.circle_bilayer(1024, radius=2.1, noise=1e-3, seed=21)
    states = {}
    for name, use, kr in (("plain", None, None), ("learned", net, None),
                          ("learned_in_training_step_range", net, (5e-4, 2e-3))):
        with fch.Context(1024, fch.params_default(0.0, zero_stab_cap=1)) as ctx:
            ctx.set_state(u0)
            t0 = time.perf_counter()
            st, trials, learned = T.run_adaptive_psd(ctx, 1e-6, args.fno_t_adaptive, dev, net=use, k_range=kr)
            ad[name] = {"wall_s": time.perf_counter() - t0, "trials": trials, "learned_trials": learned,
                        "steps": st["n_steps"], "psd_iter": st["n_psd_iter"], "t_reached": st["t"],
                        "k_last": st["k_last"]}
            states[name] = ctx.get_state()
    for name in ("learned", "learned_in_training_step_range"):
        ad[name]["rel_l2_vs_plain"] = float(np.linalg.norm(states[name] - states["plain"])
                                            / np.linalg.norm(states["plain"]))
    out["adaptive_1024"] = ad
    # inference time at 1024^2 and the PSD iteration it is traded against
    a = torch.zeros((1, 2, 1024, 1024), device=dev)
    y = torch.empty((1, 1024, 1024), device=dev)
    for _ in range(3):
        net.forward(a, y)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(10):
        net.forward(a, y)
    torch.cuda.synchronize()
    out["fno_forward_ms_1024"] = (time.perf_counter() - t0) / 10 * 1e3
    # BF16 weights with FP32 sums (inference): the same timing and the learned start
    # on the held-out trajectories
    net.set_bf16(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(10):
        net.forward(a, y)
    torch.cuda.synchronize()
    out["fno_forward_ms_1024_bf16_weights"] = (time.perf_counter() - t0) / 10 * 1e3
    out["eval_128_bf16_weights"] = evaluate(128, I.circle_bilayer(128, radius=2.1, noise=1e-3, seed=21), 30)
    # the spectral convolutions as truncated DFTs, the x DFT on the tensor cores
    net.set_bf16(2)
    for _ in range(3):
        net.forward(a, y)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(10):
        net.forward(a, y)
    torch.cuda.synchronize()
    out["fno_forward_ms_1024_truncated_dft_tensor_cores"] = (time.perf_counter() - t0) / 10 * 1e3
    out["eval_128_truncated_dft"] = evaluate(128, I.circle_bilayer(128, radius=2.1, noise=1e-3, seed=21), 30)
    out["eval_1024_truncated_dft"] = evaluate(1024, I.circle_bilayer(1024, radius=2.1, noise=1e-3, seed=21), 8)
    net.set_bf16(False)
    return out


def error_budget(args):
    """Per-field error of each precision against the FP64 oracle (the benchmark spec's mixed-
    precision budget) on the random bilayer network (critical parameters) at 1024^2
    and 2048^2: F(u) of the initial data; u, F(u), mass and energy after one and after
    budget_steps fixed IMEX steps of budget_dt (one step at 2048^2); SAV's u and r after
    one step; the LTE estimate e and the state after the backward-Euler start and one
    adaptive IMEX trial (Sec. 3.2). Each cell is the relative error against the oracle;
    the GPU's own FP64 mode is a second column."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2006_04784_gb300 import build as B
    B.build()
    O.build()
    from paper_2006_04784_gb300 import fch
    from paper_2006_04784_gb300 import inputs as I

    dev = torch.device("cuda", 0)
    L = 4 * math.pi
    out = {"dt": args.budget_dt, "runs": []}
    for n, nsteps in ((1024, args.budget_steps), (2048, 1)):
        u0 = I.random_network(n, d=0.75, seed=3)
        p0 = fch.params_default(0.0, eta2=0.15)
        p0.zeta, p0.D0 = 1.1, 170.0  # explicit SAV constants, the same on both sides
        op = O.params(eps=p0.eps, q=p0.q, gamma=p0.gamma, eta1=p0.eta1, eta2=p0.eta2, zeta=p0.zeta,
                      D0=p0.D0, beta1=p0.beta1, beta2=p0.beta2, kappa0=p0.kappa0, kappa2=p0.kappa2)
        t0 = time.perf_counter()
        ref = {"F0": O.rhs(op, u0, L)}
        s = O.Stepper(n, L, op)
        s.set_state(u0)
        for k in range(nsteps):
            s.step("imex", args.budget_dt)
            if k == 0:
                ref["u1"] = s.state()
        ref["uN"] = s.state()
        ref["FN"] = O.rhs(op, ref["uN"], L)
        ref["mass"], ref["energy"] = O.mass(ref["uN"], L), O.energy(op, ref["uN"], L)
        s = O.Stepper(n, L, op)
        s.set_state(u0)
        s.step("sav", args.budget_dt)
        ref["sav_u"], ref["sav_r"] = s.state(), s.r(0)
        s = O.Stepper(n, L, op)
        s.set_state(u0)
        s.adaptive_begin("imex", SIGMA, T_FINAL)
        s.adaptive_trial()
        ref["lte_e"], ref["ad_u"] = s.last_e, s.state()
        oracle_s = time.perf_counter() - t0
        res = {}
        for name, prec in (("fp64", fch.FCH_FP64), ("fp32x2", fch.FCH_FP32X2), ("fp32", fch.FCH_MIXED)):
            p = fch.params_default(0.0, eta2=0.15, prec=prec)
            p.zeta, p.D0 = p0.zeta, p0.D0
            r = {}
            with fch.Context(n, p) as ctx:
                def rhs(u):
                    ut = torch.tensor(u, device=dev)
                    F = torch.empty_like(ut)
                    torch.cuda.synchronize()
                    ctx.rhs_device(ut, F)
                    ctx.synchronize()
                    return F.cpu().numpy()
                r["F0"] = rhs(u0)
                ctx.set_state(u0)
                for k in range(nsteps):
                    ctx.step("imex", args.budget_dt)
                    if k == 0:
                        r["u1"] = ctx.get_state()
                r["uN"] = ctx.get_state()
                r["FN"] = rhs(r["uN"])
                r["mass"], r["energy"] = ctx.mass(), ctx.energy()
                ctx.set_state(u0)
                ctx.step("sav", args.budget_dt)
                r["sav_u"], r["sav_r"] = ctx.get_state(), ctx.sav_r()[0]
                ctx.set_state(u0)
                ctx.adaptive_begin("imex", SIGMA, T_FINAL)
                ctx.adaptive_enqueue(1)
                st = ctx.adaptive_end()
                r["lte_e"], r["ad_u"] = st["e_last"], ctx.get_state()
            res[name] = r

        def errs(a, b):
            e = {}
            for f in ("F0", "u1", "uN", "FN", "sav_u", "ad_u"):
                e[f] = _rel(a[f], b[f])
            for f in ("mass", "energy", "sav_r", "lte_e"):
                e[f] = abs(a[f] - b[f]) / abs(b[f])
            return e

        row = {"n": n, "steps": nsteps, "oracle_s": oracle_s,
               "fields": {"F0": "F(u0)", "u1": "u after 1 IMEX step", "uN": f"u after {nsteps} IMEX steps",
                          "FN": f"F(u) after {nsteps} steps", "mass": f"mass after {nsteps} steps",
                          "energy": f"energy after {nsteps} steps", "sav_u": "u after 1 SAV step",
                          "sav_r": "SAV r after 1 step", "lte_e": "LTE estimate e of the first trial",
                          "ad_u": "u after the start and one adaptive trial"}}
        for name in ("fp64", "fp32x2", "fp32"):
            row[name] = {"vs_oracle": errs(res[name], ref)}
            if name != "fp64":
                row[name]["vs_gpu_fp64"] = errs(res[name], res["fp64"])
        out["runs"].append(row)
    return out


def run_reference(args):
    """The oracle as the reference arm: adaptive IMEX trials at 1024^2 on the host
    cores, each step one trial (bounded: at most ~150 s of timed work). The workload
    (config) is the GPU arm's; the oracle computes it in FP64 whatever --prec says."""
    rank, world, _ = rank_info()
    if rank != 0:
        return None
    import numpy as np

    from oracle import oracle as O
    from paper_2006_04784_gb300 import inputs as I

    O.build()
    n = N_GRID
    L = 4 * math.pi
    u0 = I.random_network(n, d=0.75, seed=3)
    s = O.Stepper(n, L, O.params(eta2=0.15, zeta=1.1, D0=170.0))
    s.set_history(u0, u0, 1e-6)
    s.run_adaptive("imex", SIGMA, T_FINAL, max_attempts=max(1, min(args.warmup, 3)))
    K = args.steps
    t0 = time.perf_counter()
    done = 0
    while done < K:
        s.run_adaptive("imex", SIGMA, T_FINAL, max_attempts=1)
        done += 1
        if time.perf_counter() - t0 > 150:
            break
    dt = time.perf_counter() - t0
    v = done / dt
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": world,
            "steps": done, "warmup": args.warmup, "ms_per_step": 1e3 * dt / done,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded random bilayer network, no dataset)",
            "config": dict(config(args.prec), parallelism="single"),
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"{done} adaptive IMEX trials at 1024^2 (of {K} asked; "
                                       "capped at 150 s), FP64 oracle, one thread"},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--prec", default="fp32x2", choices=["mixed", "fp64", "fp32x2"],
                    help="mixed (single-precision transforms), fp64, or fp32x2 (double-float)")
    ap.add_argument("--scheme", default="imex", choices=["imex", "sav", "etd"])
    ap.add_argument("--no-t-final", action="store_true", help="skip the time-to-t_final runs")
    ap.add_argument("--no-fft", action="store_true", help="skip the standalone transform throughput")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched-ensemble entry")
    ap.add_argument("--autotune", type=int, default=2,
                    help="2: pass tiles from fch_autotune_step (timed on adaptive trials; default); "
                         "1: from fch_autotune (timed on transforms); 0: default tiles")
    ap.add_argument("--paper-costs", action="store_true",
                    help="run the Sec. 5.2 cost comparison (super-critical benchmark) instead")
    ap.add_argument("--paper-T", type=float, default=250.0)
    ap.add_argument("--comp-error", action="store_true",
                    help="the cross-scheme differences of Table t:Comp-error (five benchmarks) instead")
    ap.add_argument("--dollars-per-digit", action="store_true",
                    help="global error and transforms against sigma_tol (Sec. 5.2) for one benchmark instead")
    ap.add_argument("--dpd-benchmark", default="supercritical", choices=sorted(PAPER_REFERENCE))
    ap.add_argument("--traces", action="store_true",
                    help="global error, step size and far-field traces over time on one benchmark instead")
    ap.add_argument("--trace-benchmark", default="supercritical", choices=sorted(PAPER_T))
    ap.add_argument("--dpd-sigmas", default="", help="comma-separated sigma_tol values of the sweep")
    ap.add_argument("--dpd-etd-min", type=float, default=1e-6, help="smallest sigma_tol of the ETD sweep")
    ap.add_argument("--dpd-psd-min", type=float, default=1e-7, help="smallest sigma_tol of the PSD sweep")
    ap.add_argument("--psd-max-iter", type=int, default=1000,
                    help="PSD iterations per step before FCH_ENOCONV in the paper-benchmark modes")
    ap.add_argument("--workloads", action="store_true",
                    help="measure the 128^2 fixed-step, 512^2 all-scheme and 1024^2/2048^2 runs instead")
    ap.add_argument("--workload-t2", type=float, default=50.0)
    ap.add_argument("--workload-t3", type=float, default=10.0)
    ap.add_argument("--workload-budget", type=int, default=400000)
    ap.add_argument("--ensemble", action="store_true",
                    help="the 64-instance uneven-grid ensemble against sequential runs instead")
    ap.add_argument("--ensemble-t", type=float, default=0.02)
    ap.add_argument("--ensemble-rounds", type=int, default=8)
    ap.add_argument("--ensemble-autotune", type=int, default=2, choices=[0, 1, 2],
                    help="pass tiles of the ensemble's members (as fch_params.autotune)")
    ap.add_argument("--fno", action="store_true",
                    help="train the FNO initial iterate and compare PSD started from it instead")
    ap.add_argument("--fno-steps", type=int, default=60)
    ap.add_argument("--fno-iters", type=int, default=1500)
    ap.add_argument("--fno-lr", type=float, default=1e-3)
    ap.add_argument("--fno-t-adaptive", type=float, default=2e-2)
    ap.add_argument("--fno-forward-n", type=int, default=0,
                    help="--fno-forward: one grid size only (0: 128, 256, 512, 1024)")
    ap.add_argument("--fno-forward-mode", type=int, default=-1,
                    help="--fno-forward: one mode only (0 FP32, 1 bf16 weights, 2 tensor cores; -1: all)")
    ap.add_argument("--fno-forward", action="store_true",
                    help="only the FNO forward pass time per grid and mode (FP32, BF16 weights, truncated DFTs)")
    ap.add_argument("--fft-only", action="store_true",
                    help="only the standalone transform throughput (fch_fft_r2c / c2r against cuFFT)")
    ap.add_argument("--fft-batch", type=int, default=32)
    ap.add_argument("--fft-iters", type=int, default=10)
    ap.add_argument("--error-budget", action="store_true",
                    help="per-field single/double-float vs FP64 errors at 1024^2 and 2048^2 instead")
    ap.add_argument("--budget-steps", type=int, default=5)
    ap.add_argument("--budget-dt", type=float, default=1e-6)
    args = ap.parse_args()
    PSD_MAX_ITER[0] = args.psd_max_iter
    if args.paper_costs:
        out = paper_costs(args)
    elif args.comp_error:
        out = comp_error(args)
    elif args.dollars_per_digit:
        out = dollars_per_digit(args)
    elif args.traces:
        out = traces(args)
    elif args.workloads:
        out = workloads(args)
    elif args.error_budget:
        out = error_budget(args)
    elif args.fft_only:
        out = fft_only(args)
    elif args.fno_forward:
        out = fno_forward_times(args)
    elif args.ensemble:
        out = ensemble_bench(args)
    elif args.fno:
        out = fno_bench(args)
    else:
        out = run_reference(args) if args.impl == "reference" else run_gb300(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
