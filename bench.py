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


TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "fused_chi2_fp32_64ant.traffic.txt")


def profiled_traffic():
    """DRAM bytes per launch of the fused chi^2 kernel from the committed ncu
    record (key: value lines), or None when the kernel source changed since
    the capture."""
    import hashlib
    try:
        text = open(TRAFFIC_RECORD).read()
        src = open(os.path.join(ROOT, "paper_1501_07719_gb300", "csrc", "rime_fused.cu"), "rb").read()
    except OSError:
        return None
    vals = dict(line.split(": ", 1) for line in text.splitlines()
                if line.startswith(("traffic_bytes_per_launch: ", "source_md5: ")))
    if "traffic_bytes_per_launch" not in vals or "source_md5" not in vals:
        return None
    if not vals["source_md5"].startswith(hashlib.md5(src).hexdigest()[:12]):
        return None
    return int(vals["traffic_bytes_per_launch"])


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


def _events(torch, n):
    return [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]


def _timed(torch, stream, fn, reps):
    """Median device time (ms) of fn() over reps calls, events on the stream."""
    ev = _events(torch, reps)
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ev)


def form_small_latency(torch, R):
    """The 7-antenna, 10-timestep, 16-channel, 10-point FP64 workload (3360
    visibilities): latency-bound, so the time of one chi^2 replayed from a
    CUDA graph (result left on the device) is the number that matters."""
    wl = rime_synth.WORKLOADS["7ant-10t-16ch-10pt"]
    inp = rime_synth.make_inputs(wl, precision="f64")
    stream = torch.cuda.Stream()
    ctx = R.Rime(inp, R.RIME_FP64, weight=inp["weight"], stream=stream)
    ctx.set_gains(inp["gains"])
    ctx.set_sources(inp["sources"])
    V = ctx.predict()
    ctx.set_data(V.cpu().numpy() + inp["noise"], inp["weight"])
    del V
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.chi2_async(out)
    ctx.sync()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        g.capture_begin(capture_error_mode="relaxed")
        for _ in range(100):
            ctx.chi2_async(out)
        g.capture_end()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):   # replays run on the current stream
        g.replay()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(10):
            g.replay()
        e1.record()
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / 1000
    eager = _timed(torch, stream, lambda: ctx.chi2_async(out), 50) * 1e3
    ctx.close()
    return {"workload": wl.name, "dtype": "f64", "us_per_chi2_graph": us,
            "us_per_chi2_eager_call": eager, "eager_note": "one rime_chi2_async call per chi^2 from Python; "
            "the gap between calls is host time",
            "chi2_evals_per_s": 1e6 / us}


def form_sampler(torch, R):
    """Ensemble Metropolis over the batched observation (64 antennas, 50 t,
    32 ch): 128 chains on the 100-source sky model, each moving l, m, I and
    alpha of its brightest source, the proposal widths adapted during burn-in
    towards 30 % acceptance. Scored two ways: the 128 whole proposed sky
    models (128 x 100 sources) in one batched chi^2 call per step, and the
    moved source against per-chain residuals held on the GPU (rime_chains_*:
    the predict of 2 sources per chain per step)."""
    from paper_1501_07719_gb300 import sampler
    wl = rime_synth.WORKLOADS["64ant-50t-32ch-512sets"]
    inp = rime_synth.make_inputs(wl, precision="f32")
    w = inp["weight"].astype(np.float32)
    ctx = R.Rime(inp, R.RIME_FP32, weight=w)
    ctx.set_gains(inp["gains"])
    ctx.set_sources(inp["sources"])
    V = ctx.predict()
    ctx.set_data((V.cpu().numpy().astype(np.complex128) + inp["noise"]).astype(np.complex64), w)
    del V
    one = np.zeros(wl.nsrc)
    one[int(np.argmax(inp["sources"]["stokes"][:, 0]))] = 1.0
    steps = {"l": 1e-9 * one, "m": 1e-9 * one, "I": 1e-4 * one, "alpha": 1e-4 * one}
    out = {"workload": wl.name + " observation, 100-source sky model", "chains": 128,
           "params_moved_per_chain": 4}
    for mode, delta in (("batched", False), ("delta", True)):
        s = sampler.EnsembleMetropolis(ctx, inp["sources"], 128, steps, seed=1, delta=delta)
        scale = s.adapt(24, target=0.3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = s.run(8)
        dt = (time.perf_counter() - t0) / 8
        out[mode] = {"seconds_per_step": dt, "proposals_per_s": 128 / dt,
                     "accept_rate": float(res["accept"].mean()), "adapted_step_scale": float(scale[-1])}
    ctx.close()
    out["delta_speedup"] = out["batched"]["seconds_per_step"] / out["delta"]["seconds_per_step"]
    out["note"] = ("wall clock per step: host proposals, scoring, accept/reject; batched: one rime_chi2_batched "
                   "call (128 sets x 100 sources); delta: rime_chains_propose (2 sources per chain against its "
                   "residual D - V, 128 x 103 MB resident) and rime_chains_accept for the accepted chains; "
                   "24 burn-in steps adapt the proposal widths towards 30 % acceptance")
    return out


def _grad_times(torch, R, wl, precision, reps):
    """(chi^2 + gradient ms, plain chi^2 ms) of one workload in one precision."""
    f64 = precision == "f64"
    inp = rime_synth.make_inputs(wl, precision=precision)
    w = inp["weight"] if f64 else inp["weight"].astype(np.float32)
    ctx = R.Rime(inp, R.RIME_FP64 if f64 else R.RIME_FP32, weight=w)
    ctx.set_gains(inp["gains"])
    ctx.set_sources(inp["sources"])
    V = ctx.predict()
    D = V.cpu().numpy().astype(np.complex128) + inp["noise"]
    del V
    ctx.set_data(D if f64 else D.astype(np.complex64), w)
    stream = torch.cuda.current_stream()
    gs = torch.zeros((wl.nsrc, 10), dtype=torch.float64, device="cuda")
    gg = torch.zeros((wl.ntime, wl.na, wl.nchan, 2, 2), dtype=torch.complex128, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    R.rime_chi2_grad(ctx.ctx, gs, gg)
    if not f64:
        R.rime_chi2_grad(ctx.ctx, gs, gg)
    grad_ms = _timed(torch, stream, lambda: R.rime_chi2_grad(ctx.ctx, gs, gg), reps)
    ctx.chi2_async(out)
    plain_ms = _timed(torch, stream, lambda: ctx.chi2_async(out), 4 * reps)
    ctx.close()
    return grad_ms, plain_ms


def form_grad(torch, R, chi2_ms):
    """Adjoint gradient (rime_chi2_grad) on the 64-antenna gradient workload,
    against the plain fused chi^2 of the same workload, in FP32 (the top-level
    keys) and FP64."""
    wl = rime_synth.WORKLOADS["64ant-100t-64ch-100pt100g-grad"]
    grad_ms, plain_ms = _grad_times(torch, R, wl, "f32", 5)
    g64, p64 = _grad_times(torch, R, wl, "f64", 2)
    nparam = 10 * wl.nsrc
    return {"workload": wl.name, "dtype": "f32", "chi2_grad_ms": grad_ms, "chi2_ms": plain_ms,
            "grad_over_chi2": grad_ms / plain_ms,
            "speedup_vs_central_fd_of_source_params": 2 * nparam * plain_ms / grad_ms,
            "f64": {"chi2_grad_ms": g64, "chi2_ms": p64, "grad_over_chi2": g64 / p64},
            "fd_basis": f"central differences need 2 x {nparam} chi^2 evaluations for the source "
                        "parameters alone; the adjoint also returns the gains gradient",
            "outputs": "chi^2, d/d(l, m, I, Q, U, V, alpha, major, minor, pa) per source, d/dG per "
                       "(t, antenna, channel, Jones entry)"}


def form_batched(torch, R):
    """Batched chi^2 of 512 sky models (5..500 sources each) against one shared
    observation: one persistent launch replayed from a CUDA graph, against 512
    plain rime_chi2_async calls (one per set) on the same GPU."""
    wl = rime_synth.WORKLOADS["64ant-50t-32ch-512sets"]
    inp = rime_synth.make_inputs(wl, precision="f32")
    sets = inp["sets"]
    off = sets["offsets"]
    nsets = len(off) - 1
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    w = inp["weight"].astype(np.float32)
    ctx = R.Rime(inp, R.RIME_FP32, weight=w, stream=stream)
    ctx.set_gains(inp["gains"])
    ctx.set_sources(inp["sources"])          # the 100-source truth sky
    V = ctx.predict()
    ctx.set_data((V.cpu().numpy().astype(np.complex128) + inp["noise"]).astype(np.complex64), w)
    del V
    dev = {k: torch.tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda")
           for k, v in sets["sources"].items()}
    out = torch.zeros(nsets, dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    ctx.chi2_batched(off, dev, out=out)      # buffers + tuning trials
    ctx.sync()
    first_s = time.perf_counter() - t0
    cfg = ctx.batched_config()
    g = torch.cuda.CUDAGraph()
    g.capture_begin(capture_error_mode="relaxed")
    ctx.chi2_batched(off, dev, out=out)
    g.capture_end()
    g.replay()
    torch.cuda.synchronize()
    batched_ms = _timed(torch, stream, g.replay, 3)
    ref = out.cpu().numpy().copy()
    outp = torch.zeros(nsets, dtype=torch.float64, device="cuda")
    views = [{k: v[off[j]:off[j + 1]] for k, v in dev.items()} for j in range(nsets)]

    def plain():
        for j in range(nsets):
            ctx.set_sources(views[j])
            ctx.chi2_async(outp[j:j + 1])
    plain()
    plain_ms = _timed(torch, stream, plain, 2)
    rel = np.abs(outp.cpu().numpy() - ref) / ref
    ctx.close()
    torch.cuda.set_stream(torch.cuda.default_stream())
    isg = sets["sources"]["shape"][:, 0] > 0
    flops = (FLOPS_POINT * int((~isg).sum()) + FLOPS_GAUSS * int(isg.sum())) * wl.ntime * wl.nbl * wl.nchan
    return {"workload": wl.name, "dtype": "f32 visibilities, f64 chi^2", "nsets": nsets,
            "set_nsrc": [int(np.diff(off).min()), int(np.diff(off).max())], "total_sources": int(off[-1]),
            "batched_ms": batched_ms, "plain_512_calls_ms": plain_ms, "speedup_vs_plain": plain_ms / batched_ms,
            "chi2_evals_per_s": nsets / (batched_ms * 1e-3),
            "tflops": flops / (batched_ms * 1e-3) / 1e12, "first_call_s_incl_tuning": first_s,
            "max_rel_diff_vs_plain": float(rel.max()),
            "launch": "captured CUDA graph: schedule upload, source prep, one persistent kernel, per-set sums",
            "tuned": {k: cfg[k] for k in ("channels_per_item", "blocks_per_sm", "order", "sets_per_item", "tuned")},
            "trials_ms": [round(t["ms"], 3) for t in cfg["trials"]]}


def form_split(torch, R):
    """Point-source sum as split-precision tcgen05 MMAs (BF16 and TF32 hi+lo)
    on the 256-antenna, 4096-point workload, against the plain FP32 direct
    sum; errors against the FP64 oracle on sampled visibilities and, for
    chi^2, on a one-timestep, two-channel slice of the same workload."""
    import oracle
    wl = rime_synth.WORKLOADS["256ant-20t-128ch-4096pt"]
    inp = rime_synth.make_inputs(wl, precision="f32")
    w = inp["weight"].astype(np.float32)
    ctx = R.Rime(inp, R.RIME_FP32, weight=w)
    ctx.set_gains(inp["gains"])
    ctx.set_sources(inp["sources"])
    V = ctx.predict()
    D = (V.cpu().numpy().astype(np.complex128) + inp["noise"]).astype(np.complex64)
    del V
    ctx.set_data(D, w)
    stream = torch.cuda.current_stream()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(1)   # the samples of the split parity test
    n = 192
    t, bl, k = rng.integers(0, wl.ntime, n), rng.integers(0, wl.nbl, n), rng.integers(0, wl.nchan, n)
    p, q = rime_synth.baseline_pairs(wl.na)
    vref = oracle.Problem(inp).vis_list(t, p[bl], q[bl], k)
    # the chi^2 slice: timestep 0, channels 0-1, data = the oracle's model +
    # the workload's noise (so that V - D is the noise for an exact model)
    sl = dict(inp, ntime=1, nchan=2, freq=inp["freq"][:2], uvw=inp["uvw"][:1],
              gains=inp["gains"][:1, :, :2], weight=w[:1, :, :2])
    Dsl = np.ascontiguousarray(rime_synth.observe(oracle.Problem(sl).predict(), inp["noise"][:1, :, :2], "f32"))
    chi_ref = oracle.Problem(sl, data=Dsl).chi2()
    csl = R.Rime(sl, R.RIME_FP32, data=Dsl, weight=np.ascontiguousarray(w[:1, :, :2]))
    csl.set_gains(np.ascontiguousarray(inp["gains"][:1, :, :2]))
    csl.set_sources(inp["sources"])
    res = {}
    for mode, name in ((R.RIME_TC_OFF, "direct_fp32"), (R.RIME_TC_SPLIT_BF16, "split_bf16"),
                       (R.RIME_TC_SPLIT_TF32, "split_tf32"), (R.RIME_TC_SPLIT_F16, "split_f16")):
        ctx.set_tensor_mode(mode)
        ctx.chi2_async(out)
        ms = _timed(torch, stream, lambda: ctx.chi2_async(out), 2 if mode == R.RIME_TC_OFF else 5)
        V = ctx.predict()
        idx = [torch.tensor(a, device="cuda") for a in (t, bl, k)]
        got = V[idx[0], idx[1], idx[2]].cpu().numpy().astype(np.complex128)
        del V
        torch.cuda.empty_cache()
        csl.set_tensor_mode(mode)
        chi_sl = csl.chi2()
        res[name] = {"ms": ms, "vis_err_vs_fp64": float(np.abs(got - vref).max() / np.abs(vref).max()),
                     "chi2_rel_err_vs_fp64": abs(chi_sl - chi_ref) / chi_ref}
    ctx.close()
    csl.close()
    # roofline of the split kernels: algorithmic tensor flops = the real products
    # the baselines need (nbl x nsrc x 4 Stokes x 2 parts x K=2 per source x 2
    # flops) times the three split products, against the measured sustained
    # BF16 peak (TF32: times the nominal TF32/BF16 ratio 1.1/2.25)
    pk = measured_peaks()
    bf16_peak = pk.get("bf16_tflops_sustained", 1700.0)
    algo = wl.ntime * wl.nchan * wl.nbl * wl.nsrc * 4 * 2 * 2 * 2 * 3
    for name, peak in (("split_bf16", bf16_peak), ("split_tf32", bf16_peak * 1.1 / 2.25), ("split_f16", bf16_peak)):
        res[name]["speedup_vs_direct"] = res["direct_fp32"]["ms"] / res[name]["ms"]
        ach = algo / (res[name]["ms"] * 1e-3) / 1e12
        res[name]["roofline"] = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                                 "frac": ach / peak,
                                 "peak_basis": "MEASURED_PEAKS.json bf16_tflops_sustained"
                                 + (" x 1.1/2.25 (nominal TF32/BF16)" if name == "split_tf32" else "")}
    res["workload"] = wl.name
    res["terms_per_s"] = {kk: terms_of(wl) / (v["ms"] * 1e-3) for kk, v in res.items() if isinstance(v, dict)}
    res["errors"] = ("vis: max |V - V_fp64| / max |V_fp64| over 192 sampled (t, baseline, channel); "
                     "chi2: |chi2 - chi2_fp64| / chi2_fp64 on timestep 0, channels 0-1, data = the FP64 model + noise")
    return res


# Table 4: Montblanc's time (s) on a K40 for the full RIME + chi^2 at 64
# channels, 100 timesteps, 50 point + 50 Gaussian sources: (FP32, FP64).
K40_TABLE4_S = {7: (0.0042, 0.0073), 14: (0.0136, 0.0215), 27: (0.0435, 0.0703), 64: (0.2320, 0.3668),
                128: (0.7007, 0.9113), 192: (1.5730, 2.3540)}


def _sweep_time(torch, R, wl, f64, reps, grad=False):
    """Median device time (ms) of one fused chi^2 on workload wl (and, with
    grad, of one chi^2 + gradient call); the data are zero and the weights
    the workload's (the cost does not depend on values)."""
    inp = rime_synth.make_inputs(wl, precision="f64" if f64 else "f32", noise=False)
    cdt = torch.complex128 if f64 else torch.complex64
    rdt = np.float64 if f64 else np.float32
    stream = torch.cuda.current_stream()
    D = torch.zeros((wl.ntime, wl.nbl, wl.nchan, 4), dtype=cdt, device="cuda")
    W = torch.from_numpy(inp["weight"].astype(rdt)).cuda()
    ctx = R.Rime(inp, R.RIME_FP64 if f64 else R.RIME_FP32, data=D, weight=W, stream=stream)
    del D, W
    ctx.set_gains(inp["gains"])
    ctx.set_sources(inp["sources"])
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        ctx.chi2_async(out)
    ctx.sync()
    ms = _timed(torch, stream, lambda: ctx.chi2_async(out), reps)
    if grad:
        gs = torch.zeros((wl.nsrc, 10), dtype=torch.float64, device="cuda")
        gg = torch.zeros((wl.ntime, wl.na, wl.nchan, 2, 2), dtype=torch.complex128, device="cuda")
        R.rime_chi2_grad(ctx.ctx, gs, gg)
        gms = _timed(torch, stream, lambda: R.rime_chi2_grad(ctx.ctx, gs, gg), max(2, reps // 3))
        ctx.close()
        return ms, gms
    ctx.close()
    return ms


def form_sweep(torch, R):
    """The paper's problem-size studies on synthetic inputs of the same shapes:
    (1) Table 4's antenna sweep (7-192 antennas, 100 timesteps, 64 channels,
    50 point + 50 Gaussian sources) in FP32 and FP64, next to the paper's K40
    times; (2) the dimension variation of Sec. 5 (the 7-antenna case with the
    channels, timesteps, point or Gaussian sources multiplied), as device time
    per source-term, which shows what a unit of each dimension costs."""
    rows = []
    for na in sorted(K40_TABLE4_S):
        wl = rime_synth.custom(na, 100, 64, 50, 50, seed_index=200 + na)
        row = {"na": na, "nbl": wl.nbl}
        for i, (name, f64) in enumerate((("f32", False), ("f64", True))):
            reps = 3 if (f64 and na >= 128) else 10
            if f64:
                ms = _sweep_time(torch, R, wl, f64, reps)
            else:
                ms, gms = _sweep_time(torch, R, wl, f64, reps, grad=True)
            row[name] = {"ms": ms, "terms_per_s": terms_of(wl) / (ms * 1e-3),
                         "k40_s": K40_TABLE4_S[na][i], "speedup_vs_k40": K40_TABLE4_S[na][i] / (ms * 1e-3)}
            if not f64:
                row[name]["chi2_grad_ms"] = gms
                row[name]["grad_over_chi2"] = gms / ms
        rows.append(row)
    base = dict(na=7, ntime=100, nchan=64, npsrc=50, ngsrc=50)
    dims = {"nchan": [64, 128, 256, 512], "ntime": [100, 300, 600, 1000],
            "npsrc": [50, 550, 1150, 1950], "ngsrc": [50, 550, 1150, 1950]}
    var = {}
    for dim, vals in dims.items():
        pts = []
        for v in vals:
            kw = dict(base, **{dim: v})
            wl = rime_synth.custom(kw["na"], kw["ntime"], kw["nchan"], kw["npsrc"], kw["ngsrc"], seed_index=260)
            ms = _sweep_time(torch, R, wl, False, 10)
            pts.append({dim: v, "ms": ms, "source_terms": terms_of(wl) // 4,
                        "ns_per_source_term": ms * 1e6 / (terms_of(wl) // 4)})
        var[dim] = pts
    return {"antennas": {"workload": "N ant, 100 t, 64 ch, 50 pt + 50 gauss (Table 4 shapes)",
                         "rows": rows},
            "dimension_variation": {"workload": "7 ant, 100 t, 64 ch, 50 pt + 50 gauss, one dimension "
                                                "multiplied (Sec. 5 dimension study), FP32", "series": var},
            "note": "device time of one fused chi^2 (CUDA events, median); the K40 times are the paper's "
                    "Table 4 (full RIME + chi^2 on a K40), context not target"}


def form_peaks(torch, R):
    """Measured issue rates of the FP32 (scalar and packed), FP64 and SFU
    pipes (rime_pipe_rate), with the SM clock sampled while they run: the
    denominators of the ALU rooflines."""
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    time.sleep(0.2)
    rates = {name: R.rime_pipe_rate(pipe) for name, pipe in
             (("ffma", R.RIME_PIPE_FFMA), ("ffma2", R.RIME_PIPE_FFMA2), ("dfma", R.RIME_PIPE_DFMA),
              ("ex2", R.RIME_PIPE_EX2))}
    clocks = clk.stop()
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    per_clk = {k: v / (SM_COUNT * mhz * 1e6) for k, v in rates.items()}
    return {"lane_ops_per_s": rates, "per_sm_per_clock": per_clk, "clocks": clocks,
            "note": "one FMA counts one lane operation (a packed pair two); flops = 2 x FMA rate"}


def form_fp64(torch, R):
    """The FP64 fused chi^2 of the benchmark workload: time, terms/s and its
    roofline against the measured FP64 FMA rate."""
    wl = rime_synth.WORKLOADS[WORKLOAD]
    ms = _sweep_time(torch, R, wl, True, 3)
    dfma = R.rime_pipe_rate(R.RIME_PIPE_DFMA)
    peak = 2.0 * dfma / 1e12
    ach = algo_flops(wl) / (ms * 1e-3) / 1e12
    return {"workload": wl.name, "dtype": "f64", "ms": ms, "terms_per_s": terms_of(wl) / (ms * 1e-3),
            "roofline": {"bound": "alu", "kernel": "k_fused_f64<chi2>", "achieved": ach, "peak": peak,
                         "unit": "TFLOP/s", "frac": ach / peak,
                         "peak_basis": "measured FP64 FMA rate (rime_pipe_rate) x 2 flops",
                         "algorithmic": f"{FLOPS_POINT} flops/point term, {FLOPS_GAUSS}/Gaussian term"}}


def run_only(args):
    """One form on one (possibly reduced) workload, for profiling: prints the
    median launch time. Not the benchmark line."""
    import torch
    import paper_1501_07719_gb300 as R
    over = {k: v for k, v in (("ntime", args.ntime), ("nchan", args.nchan)) if v}
    wl = rime_synth.workload(args.workload, **over)
    f64 = args.precision == "f64"
    inp = rime_synth.make_inputs(wl, precision=args.precision)
    w = inp["weight"].astype(np.float64 if f64 else np.float32)
    stream = torch.cuda.current_stream()
    ctx = R.Rime(inp, R.RIME_FP64 if f64 else R.RIME_FP32, weight=w, stream=stream)
    ctx.set_gains(inp["gains"])
    ctx.set_sources(inp["sources"])
    V = ctx.predict()
    ctx.set_data((V.cpu().numpy().astype(np.complex128) + inp["noise"]).astype(np.complex128 if f64 else np.complex64), w)
    del V
    out = torch.zeros(max(1, wl.nsets), dtype=torch.float64, device="cuda")
    if args.only in ("chi2", "split-bf16", "split-tf32", "split-f16"):
        ctx.set_tensor_mode({"chi2": R.RIME_TC_OFF, "split-bf16": R.RIME_TC_SPLIT_BF16,
                             "split-tf32": R.RIME_TC_SPLIT_TF32, "split-f16": R.RIME_TC_SPLIT_F16}[args.only])
        fn = lambda: ctx.chi2_async(out)
    elif args.only == "chains":
        # 128 chains, each proposing a move of the brightest source against
        # its resident residual (rime_chains_propose)
        K = 128
        ctx.chains_init(K)
        j = int(np.argmax(inp["sources"]["stokes"][:, 0]))
        cur = {k: np.repeat(v[j:j + 1], K, axis=0) for k, v in inp["sources"].items()}
        rng = np.random.default_rng(0)
        prop = {k: v.copy() for k, v in cur.items()}
        prop["lm"] += rng.normal(0, 1e-8, prop["lm"].shape)
        prop["stokes"] *= 1 + rng.normal(0, 1e-3, (K, 1))
        out = torch.zeros(K, dtype=torch.float64, device="cuda")
        fn = lambda: ctx.chains_propose(1, prop, cur, out=out)
    elif args.only == "grad":
        gs = torch.zeros((wl.nsrc, 10), dtype=torch.float64, device="cuda")
        gg = torch.zeros((wl.ntime, wl.na, wl.nchan, 2, 2), dtype=torch.complex128, device="cuda")
        fn = lambda: R.rime_chi2_grad(ctx.ctx, gs, gg)
    else:
        sets = inp["sets"]
        fn = lambda: ctx.chi2_batched(sets["offsets"], sets["sources"], out=out)
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    ms = _timed(torch, stream, fn, args.steps)
    ctx.sync()   # a deferred error (e.g. a split mode given Gaussian sources) raises here
    ctx.close()
    print(json.dumps({"only": args.only, "workload": wl.name, "ntime": wl.ntime, "nchan": wl.nchan,
                      "median_ms": ms}), flush=True)
    return 0


def run_reference(args, wl, rank, world):
    """The oracle (a deliberately plain FP64 CPU program) on this host's cores:
    each step a bounded sample of the workload, so the run ends within minutes."""
    if rank != 0:
        return 0
    import oracle
    inp = rime_synth.make_inputs(wl, precision="f32")
    nt, nch = oracle.threads(), 8
    vals, secs, cb = [], [], None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(wl, inp, nt, nch)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            vals.append(cb["value"])
            secs.append(dt)
    value = statistics.median(vals) if vals else cb["value"]
    cb["value"] = value
    # one step is one oracle chi^2 of the sample: its own time, not the full workload's
    ms_step = 1e3 * (statistics.mean(secs) if secs else 0.0)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "terms/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "precision": "f64 oracle", "sample": cb["sample"],
                       "step": "one oracle chi^2 of the sample (the value is the sample's terms / its time)"},
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
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the gradient, batched and split-precision comparisons")
    ap.add_argument("--only", choices=["chi2", "grad", "batched", "split-bf16", "split-tf32", "split-f16", "sweep", "chains",
                                       "peaks", "fp64"],
                    help="time one form on --workload (optionally with fewer timesteps / channels) "
                         "instead of the benchmark; for profiling")
    ap.add_argument("--ntime", type=int, default=0)
    ap.add_argument("--nchan", type=int, default=0)
    args = ap.parse_args()
    if args.only in ("sweep", "peaks", "fp64"):
        import torch
        import paper_1501_07719_gb300 as R
        fn = {"sweep": form_sweep, "peaks": form_peaks, "fp64": form_fp64}[args.only]
        print(json.dumps(fn(torch, R)), flush=True)
        return 0
    if args.only:
        return run_only(args)
    wl = rime_synth.WORKLOADS[args.workload]
    rank, world, local = dist_setup(args.gpus)
    if args.impl == "reference":
        return run_reference(args, wl, rank, world)

    import torch
    import paper_1501_07719_gb300 as R
    from paper_1501_07719_gb300 import shard
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
        total_ms = shard.reduce_max(total_ms)   # the slowest rank
    ms_per_step = total_ms / args.steps
    terms = terms_of(wl)
    value = terms * world / (ms_per_step * 1e-3)

    # ---- end to end through the public API with host buffers ----
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_uvw, h_D, h_w, h_g = pin(inp["uvw"]), pin(D), pin(weight), pin(inp["gains"])
    h_src = {k: pin(v) for k, v in inp["sources"].items()}
    h2d = sum(x.numel() * x.element_size() for x in (h_uvw, h_D, h_w, h_g, *h_src.values()))
    def e2e_step(streamed):
        # the step's inputs from pinned host memory, its chi^2 back to the host:
        # streamed, the data and weights go to the GPU in time chunks whose
        # copies overlap the kernel (rime_chi2_streamed); otherwise they are
        # uploaded whole before the kernel runs (rime_set_data + rime_chi2)
        ctx.set_uvw(h_uvw)
        ctx.set_gains(h_g)
        ctx.set_sources(h_src)
        if streamed:
            return ctx.chi2_streamed(h_D, h_w)
        ctx.set_data(h_D, h_w)
        return ctx.chi2()

    def e2e_time(streamed):
        times, chi = [], None
        for i in range(args.e2e_steps + 1):
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            chi = e2e_step(streamed)
            dt = time.perf_counter() - t0
            if i > 0:
                times.append(dt)
        s = statistics.median(times)
        return (shard.reduce_max(s) if dist else s), chi

    upload_s, chi_upload = e2e_time(False)
    e2e_s, chi_e2e = e2e_time(True)
    assert chi_upload == chi_check, (chi_upload, chi_check)
    # the streamed sum groups the same block partials per time chunk
    assert abs(chi_e2e - chi_check) <= 1e-12 * abs(chi_check), (chi_e2e, chi_check)

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
                     "frac": achieved / peak, "traffic": profiled_traffic() if args.workload == WORKLOAD else None,
                     "traffic_unit": "bytes per launch (ncu dram read + write, " + os.path.relpath(TRAFFIC_RECORD, ROOT) + ")",
                     "peak_basis": f"FP32 FMA: {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x 2 x {max_mhz:.0f} MHz",
                     "algorithmic": f"{FLOPS_POINT} flops/point term, {FLOPS_GAUSS}/Gaussian term",
                     "avg_launch_ms": avg_launch_s * 1e3},
        "e2e": {"value": terms * world / e2e_s, "unit": "terms/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": 112, "seconds_per_step": e2e_s,
                "calls": "rime_set_uvw, rime_set_gains, rime_set_sources, rime_chi2_streamed "
                         f"(chunks of {ctx.stream_chunk_ntime()} timesteps, copies overlapped with the kernel)",
                "upload_then_chi2": {"value": terms * world / upload_s, "seconds_per_step": upload_s,
                                     "calls": "rime_set_uvw, rime_set_data, rime_set_gains, rime_set_sources, "
                                              "rime_chi2 (data uploaded whole, then the kernel)"}},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "chi2": chi_check,
    }
    if clocks:
        line["roofline"]["frac_at_median_clock"] = achieved / peak_fp32_tflops(clocks["sm_mhz"])
    ctx.close()
    if rank == 0 and world == 1 and not args.no_forms and args.precision == "f32":
        line["forms"] = {"peaks": form_peaks(torch, R),
                         "fp64": form_fp64(torch, R),
                         "small_fp64_latency": form_small_latency(torch, R),
                         "gradient": form_grad(torch, R, ms_per_step),
                         "batched": form_batched(torch, R),
                         "sampler": form_sampler(torch, R),
                         "split_precision": form_split(torch, R),
                         "sweep": form_sweep(torch, R)}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, inp)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
