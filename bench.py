#!/usr/bin/env python
"""Benchmark of the fused RIME predict + chi^2 (eqs. 1-7) on one GB300.

Workload: 64 antennas (2016 baselines), 100 timesteps, 64 channels
(1.0-1.5 GHz), 100 point + 100 Gaussian sources, gains, weights, FP32
(seeded synthetic inputs shaped like the paper's Table 4 runs).

One step = one chi^2 evaluation of the whole workload (one launch of the
fused kernel: per-antenna factors, source sum, gains, residual, reduction).
Rank 0 prints one JSON line. Metric: RIME terms/s = 4 ntime nbl nchan nsrc / s.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun (N > 1) every rank evaluates its own time chunk of the same
shape (weak scaling, no data-path collective); value = all ranks' terms / max time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import rime_synth  # noqa: E402

WORKLOAD = "64ant-100t-64ch-100pt100g"
METRIC = "RIME terms/s (src x bl x chan x time x 4), fused predict + chi^2"
SM_COUNT = 152
FP32_LANES_PER_SM = 128
# algorithmic FP32 flops per source term (FMA = 2): z = A_p conj(A_q) is
# 2 mul + 2 fma (6), four Stokes accumulations are 8 fma (16); a Gaussian
# adds nu^2 * exponent (1) and z * g (2).
FLOPS_POINT, FLOPS_GAUSS = 22, 25


def peak_fp32_tflops(mhz):
    return 2.0 * FP32_LANES_PER_SM * SM_COUNT * mhz * 1e6 / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = [r.split(", ") for r in out.strip().splitlines() if r.strip()]
        rows = [r for r in rows if len(r) >= 9]
        if not rows:
            return None
        mhz = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.strip() == "Active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": float(rows[0][2]),
                "samples": len(rows), "reasons": sorted(reasons),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def dist_setup(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def terms_of(wl):
    return 4 * wl.ntime * wl.nbl * wl.nchan * wl.nsrc


def algo_flops(wl):
    return (FLOPS_POINT * wl.npsrc + FLOPS_GAUSS * wl.ngsrc) * wl.ntime * wl.nbl * wl.nchan


def cpu_baseline(wl, inp, nt=None, nch=None):
    """The FP64 oracle timed on this host's cores on a bounded sample of the same
    workload: the first nt timesteps (default 2 x threads) and nch channels (default
    all), data = noise (the oracle's cost does not depend on the data values)."""
    import oracle
    nthreads = oracle.threads()
    nt = min(wl.ntime, nt or 2 * nthreads)
    nch = min(wl.nchan, nch or wl.nchan)
    sub = dict(inp, ntime=nt, nchan=nch, freq=inp["freq"][:nch], uvw=inp["uvw"][:nt],
               gains=inp["gains"][:nt, :, :nch], weight=inp["weight"][:nt, :, :nch])
    P = oracle.Problem(sub, data=inp["noise"][:nt, :, :nch])
    t0 = time.perf_counter()
    P.chi2()
    dt = time.perf_counter() - t0
    terms = 4 * nt * wl.nbl * nch * wl.nsrc
    return {"value": terms / dt, "unit": "terms/s", "cores": nthreads, "kind": "oracle",
            "sample": f"first {nt} of {wl.ntime} timesteps x {nch} of {wl.nchan} channels "
                      f"({terms / 4:.3g} source-terms), FP64, {dt:.1f} s"}


def run_reference(args, wl, rank, world):
    """The oracle (a deliberately plain FP64 CPU program) on this host's cores:
    each step a bounded sample of the workload, so the run ends within minutes."""
    if rank != 0:
        return 0
    import oracle
    inp = rime_synth.make_inputs(wl, precision="f32")
    nt, nch = oracle.threads(), 8
    vals, cb = [], None
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(wl, inp, nt, nch)
        if i >= args.warmup:
            vals.append(cb["value"])
    value = statistics.median(vals) if vals else cb["value"]
    cb["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "terms/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": terms_of(wl) / value * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "precision": "f64 oracle", "sample": cb["sample"]},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    wl = rime_synth.WORKLOADS[args.workload]
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        return run_reference(args, wl, rank, world)

    import torch
    import paper_1501_07719_gb300 as R
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec = R.RIME_FP32 if args.precision == "f32" else R.RIME_FP64
    rd = np.float32 if args.precision == "f32" else np.float64
    cd = np.complex64 if args.precision == "f32" else np.complex128
    seed = rime_synth.SEED_BASE + wl.seed_index + 1000 * rank
    inp = rime_synth.make_inputs(wl, precision=args.precision, seed=seed)
    weight = inp["weight"].astype(rd)
    stream = torch.cuda.current_stream()
    ctx = R.Rime(inp, prec, weight=weight, stream=stream)
    ctx.set_gains(inp["gains"])
    ctx.set_sources(inp["sources"])
    # observed data: this workload's model (predicted here) plus the seeded noise
    V = ctx.predict()
    D = (V.cpu().numpy().astype(np.complex128) + inp["noise"]).astype(cd)
    del V
    ctx.set_data(D, weight)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")

    for _ in range(max(args.warmup, 3)):
        ctx.chi2_async(out)
    torch.cuda.synchronize()
    chi_check = ctx.chi2()

    # ---- device-timed region: K fused launches, events around each ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    time.sleep(0.25)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e_start.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        ctx.chi2_async(out)
        ev[i][1].record(stream)
    e_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop()
    total_ms = e_start.elapsed_time(e_end)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    if dist:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    terms = terms_of(wl)
    value = terms * world / (ms_per_step * 1e-3)

    # ---- end to end through the public API with host buffers ----
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_uvw, h_D, h_w, h_g = pin(inp["uvw"]), pin(D), pin(weight), pin(inp["gains"])
    h_src = {k: pin(v) for k, v in inp["sources"].items()}
    h2d = sum(x.numel() * x.element_size() for x in (h_uvw, h_D, h_w, h_g, *h_src.values()))
    e2e_times = []
    for i in range(args.e2e_steps + 1):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.set_uvw(h_uvw)
        ctx.set_data(h_D, h_w)
        ctx.set_gains(h_g)
        ctx.set_sources(h_src)
        chi_e2e = ctx.chi2()
        dt = time.perf_counter() - t0
        if i > 0:
            e2e_times.append(dt)
    e2e_s = statistics.median(e2e_times)
    if dist:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    assert chi_e2e == chi_check, (chi_e2e, chi_check)

    peaks = measured_peaks()
    max_mhz = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    peak = peak_fp32_tflops(max_mhz)
    avg_launch_s = statistics.mean(launch_ms) * 1e-3
    achieved = algo_flops(wl) / avg_launch_s / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": wl.name, "na": wl.na, "nbl": wl.nbl, "ntime": wl.ntime,
                   "nchan": wl.nchan, "npsrc": wl.npsrc, "ngsrc": wl.ngsrc, "gains": True,
                   "chi2_evals_per_s": world / (ms_per_step * 1e-3),
                   "l2": f"inputs larger than L2: data {D.nbytes / 1e6:.0f} MB + weights "
                         f"{weight.nbytes / 1e6:.0f} MB read per step (L2 129 MB)",
                   "parallelism": f"replicas x{world} (time chunks)" if world > 1 else "1 GPU"},
        "roofline": {"bound": "alu", "kernel": "k_fused<float, chi2>", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_basis": f"FP32 FMA: {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x 2 x {max_mhz:.0f} MHz",
                     "algorithmic": f"{FLOPS_POINT} flops/point term, {FLOPS_GAUSS}/Gaussian term",
                     "avg_launch_ms": avg_launch_s * 1e3},
        "e2e": {"value": terms * world / e2e_s, "unit": "terms/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": 112, "seconds_per_step": e2e_s,
                "calls": "rime_set_uvw, rime_set_data, rime_set_gains, rime_set_sources, rime_chi2"},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "chi2": chi_check,
    }
    if clocks:
        line["roofline"]["frac_at_median_clock"] = achieved / peak_fp32_tflops(clocks["sm_mhz"])
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, inp)
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
