#!/usr/bin/env python
"""Throughput benchmark of the room-simulator filter-and-mix path.

One step = the whole hot path over one batch: RIR cut-off (Eq. 7-9), gains
from SNRs, per-utterance FFT-size choice (Eq. 6), RIR spectra, the fused
overlap-add forward (Eq. 2), the segment fix-up, and the adjoint (gradients
for sources, RIRs and gains).  Workload: 256 utterances of 2-15 s at 16 kHz,
1 target + 0-3 noise sources, 2 microphones, RT60 0.1-0.9 s, 20 dB cut-off
(synthetic, seeded).  Metric: simulated (target) audio seconds per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "simulated audio s/sec (fwd, fwd+bwd) at 16 kHz, 1×GB300, % FFT roofline vs plain"
UNIT = "audio_s/s"
ETA_DB = 20.0
REF_BUDGET_S = 120.0     # wall time the reference arm's steps aim at
WORKLOAD = ("home-256: 256 utterances, lengths U(2,15) s at 16 kHz, 1 target + 0-3 noise "
            "sources, 2 mics 7.1 cm apart, RT60 U(0.1,0.9) s, SNR U(0,30) dB, eta 20 dB")
DATA = "synthetic: AR(2) speech stand-ins, white/AR(1) noise, exponential-decay RIRs (seeded)"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


# ---------------------------------------------------------------------------
# algorithmic work (the minimum the method does at the chosen FFT sizes)
# ---------------------------------------------------------------------------
def algorithmic_work(batch, q, L, cache=False):
    """FLOPs and HBM bytes of the forward and backward OLA kernels.

    A real N-point transform counts 2.5 N log2 N flops, a complex
    multiply-add 8.  Forward per block: I + J transforms and I*J spectrum
    products; bytes: x read once, y written once.  Backward per block:
    2I + J transforms and 2*I*J products, plus one inverse per RIR for dh;
    bytes: grad_y and x read once, grad_x written once, dh written once.
    With the spectrum cache each source block is transformed once
    for the whole step: the forward also writes its half spectrum (N/4 bin
    pairs of 16 bytes) and the backward reads it in place of x and does
    I + J transforms per block."""
    ff = fb = bf = bb = 0.0
    ff5 = bf5 = 0.0           # the same with 5 N log2 N per transform (complex-FFT count)
    J = batch.num_mics
    ri = batch.rir_index()
    for u in range(batch.num_utts):
        I = int(batch.num_sources[u])
        nx = int(batch.num_samples[u])
        m = int(q["log2_n"][u])
        N = 1 << m
        B = int(q["num_blocks"][u])
        tr = 2.5 * N * m
        mac = 8.0 * (N / 2 + 1)
        cached = cache
        nbw = (I + J) if cached else (2 * I + J)             # backward transforms per block
        spec = B * I * 4.0 * N if cached else 0.0            # bytes of the kept spectra
        ff += B * ((I + J) * tr + I * J * mac)
        fb += 4.0 * (I + J) * nx + spec
        bf += B * (nbw * tr + 2 * I * J * mac) + I * J * tr
        bb += 4.0 * (J + I) * nx + (spec if cached else 4.0 * I * nx) + 4.0 * float(np.sum(L[ri[u]:ri[u + 1]]))
        ff5 += B * ((I + J) * 2 * tr + I * J * mac)
        bf5 += B * (nbw * 2 * tr + 2 * I * J * mac) + I * J * 2 * tr
    return dict(fwd_flops=ff, fwd_bytes=fb, bwd_flops=bf, bwd_bytes=bb, fwd_flops_5n=ff5, bwd_flops_5n=bf5)


def roofline_entry(flops, nbytes, ms, p_fp32_tflops, hbm_gbs, peak_kind, traffic):
    t = ms / 1e3
    t_alu = flops / (p_fp32_tflops * 1e12)
    t_hbm = nbytes / (hbm_gbs * 1e9)
    if t_alu >= t_hbm:
        ach = flops / t / 1e12
        return {"bound": "alu", "achieved": ach, "peak": p_fp32_tflops, "unit": "TFLOP/s",
                "frac": ach / p_fp32_tflops, "traffic": traffic,
                "peak_source": f"derived: SMs x 128 FP32 lanes x 2 flops x max SM clock ({peak_kind} clock)",
                "hbm_side": {"achieved": nbytes / t / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                             "frac": nbytes / t / 1e9 / hbm_gbs, "peak_source": peak_kind}}
    ach = nbytes / t / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": hbm_gbs, "unit": "GB/s", "frac": ach / hbm_gbs,
            "traffic": traffic, "peak_source": peak_kind,
            "alu_side": {"achieved": flops / t / 1e12, "peak": p_fp32_tflops, "unit": "TFLOP/s"}}


def step_roofline(work, ms, p_fp32_tflops, hbm_gbs):
    """Whole step (forward + backward) against the roof: T_roof = max(bytes /
    HBM bandwidth, flops / FP32 peak), fraction = T_roof / measured time."""
    nbytes = work["fwd_bytes"] + work["bwd_bytes"]
    t_b = nbytes / (hbm_gbs * 1e9)
    out = {}
    for key, fl in (("", work["fwd_flops"] + work["bwd_flops"]),
                    ("_5NlogN", work["fwd_flops_5n"] + work["bwd_flops_5n"])):
        t_roof = max(t_b, fl / (p_fp32_tflops * 1e12))
        out["t_roof_ms" + key] = t_roof * 1e3
        out["frac" + key] = t_roof / (ms / 1e3)
    out["bound"] = "alu" if out["t_roof_ms"] > t_b * 1e3 else "hbm"
    return out


def _traffic_for(kernel):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    source has not changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel)
    if not d:
        return None
    h = hashlib.sha256()
    for f in d["sources"]:
        h.update(open(os.path.join(ROOT, "paper_1712_03439_gb300", "csrc", f), "rb").read())
    if h.hexdigest()[:16] != d.get("source_sha"):
        return None
    return d.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# multi-rank aggregation (replicas: every rank runs the whole workload)
# ---------------------------------------------------------------------------
def reduce_max(value, dist=None, device="cpu"):
    """Max of a per-rank scalar over all ranks (the slowest rank sets the time)."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms_max):
    """Units all ranks processed per second, timed by the slowest rank."""
    return world * units_per_rank / (ms_max / 1e3)


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if len(r) > 3 and r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if len(r) > 3 and r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows if len(r) >= 10
                          for k in range(4) if r[6 + k].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# plain per-utterance GPU path (Eq. 4 full-length FFT convolution, torch.fft)
# ---------------------------------------------------------------------------
def plain_step(torch, batch, xs, hs, snrs, gys):
    """One forward + backward of the plain path: a Python loop over
    utterances, each a full-length torch.fft convolution of every (i, j)."""
    J = batch.num_mics
    fac = 10.0 ** (-ETA_DB / 10.0)
    for u in range(batch.num_utts):
        x, h, snr, gy = xs[u], hs[u], snrs[u], gys[u]
        x = x.detach().requires_grad_(True)
        h = h.detach().requires_grad_(True)
        I, nx = x.shape
        nh = h.shape[-1]
        p = h.detach() ** 2
        pth = p.amax(-1, keepdim=True) * fac
        idx = torch.arange(nh, device=h.device)
        last = torch.where(p >= pth, idx, -1).amax(-1, keepdim=True)
        keep = (idx < torch.clamp(last + 2, max=nh)).to(h.dtype)
        hh = h * keep
        pw = (x.detach() ** 2).mean(-1)
        a = torch.sqrt(pw[0] / pw * torch.pow(10.0, -snr / 10.0))
        a = torch.cat([torch.ones_like(a[:1]), a[1:]]).requires_grad_(True)
        n = 1 << int(math.ceil(math.log2(nx + nh - 1)))
        X = torch.fft.rfft(x, n)                       # [I, F]
        H = torch.fft.rfft(hh, n)                      # [I, J, F]
        Y = torch.einsum("i,if,ijf->jf", a.to(X.dtype), X, H)
        y = torch.fft.irfft(Y, n)[:, :nx]
        (y * gy).sum().backward()
    return None


def _plain_inputs(torch, dev, b, x=None, rir=None, snr=None, gy=None):
    """Per-utterance views (sources [I, Nx], zero-padded RIRs [I, J, Nh_max],
    SNRs, upstream gradient [J, Nx]) for the plain path."""
    from paper_1712_03439_gb300 import synth
    x = torch.from_numpy(b.x).to(dev) if x is None else x
    rir = torch.from_numpy(b.rir).to(dev) if rir is None else rir
    snr = torch.from_numpy(b.snr_db).to(dev) if snr is None else snr
    gy = torch.from_numpy(synth.grad_like(99, b.y_size)).to(dev) if gy is None else gy
    xo, ro, si, ri = b.x_offsets(), b.rir_offsets(), b.src_index(), b.rir_index()
    yo = b.y_offsets()
    xs, hs, snrs, gys = [], [], [], []
    for u in range(b.num_utts):
        I, nx = int(b.num_sources[u]), int(b.num_samples[u])
        xs.append(x[xo[si[u]]:xo[si[u + 1]]].view(I, nx))
        lens = b.rir_len[ri[u]:ri[u + 1]]
        hp = torch.zeros(I * b.num_mics, int(lens.max()), device=dev)
        for k, r in enumerate(range(ri[u], ri[u + 1])):
            hp[k, :lens[k]] = rir[ro[r]:ro[r + 1]]
        hs.append(hp.view(I, b.num_mics, -1))
        snrs.append(snr[si[u]:si[u + 1]])
        gys.append(gy[yo[u]:yo[u + 1]].view(b.num_mics, nx))
    return xs, hs, snrs, gys


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on a bounded sample
# ---------------------------------------------------------------------------
def host_cpu() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample_step(oracle, sub, g):
    out = oracle.forward(sub, ETA_DB)
    oracle.backward(sub, out["L"], out["alpha"], g)


def run_reference(args):
    import oracle
    from paper_1712_03439_gb300 import synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    b = synth.config_home()
    cores = oracle.max_threads()
    # as many utterances as the oracle has threads (at least 16): its forward runs one
    # work item per (utterance, microphone) and its backward one per source, so every
    # core has work
    n_utts = min(b.num_utts, max(16, cores))
    utts = b.subset(range(n_utts))
    # the sample per step: the first T seconds of those utterances (all sources, whole RIRs),
    # T chosen from a one-second calibration so that the K + W steps take about REF_BUDGET_S
    # (the direct form's cost grows linearly with T)
    cal = utts.excerpt(synth.FS)
    g_cal = synth.grad_like(99, cal.y_size)
    t0 = time.perf_counter()
    oracle_sample_step(oracle, cal, g_cal)
    t_one = time.perf_counter() - t0
    per_step = REF_BUDGET_S / max(args.steps + args.warmup, 1)
    n = int(min(utts.num_samples.max(), max(0.25 * synth.FS, synth.FS * per_step / max(t_one, 1e-6))))
    sub = utts.excerpt(n)
    g = synth.grad_like(99, sub.y_size)
    for _ in range(args.warmup):
        oracle_sample_step(oracle, sub, g)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_sample_step(oracle, sub, g)
    dt = (time.perf_counter() - t0) / args.steps
    v = sub.audio_seconds() / dt
    sample = (f"the first {n / synth.FS:.2f} s of utterances 0-{n_utts - 1} of the home-256 batch "
              f"({sub.audio_seconds():.2f} s of audio, {int(sub.num_sources.sum())} sources, whole RIRs), "
              f"forward + backward, direct FP64 on {cores} threads of {host_cpu()}; "
              f"the excerpt length keeps the run near {REF_BUDGET_S:.0f} s")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": DATA, "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "nproc": os.cpu_count(), "cpu_model": host_cpu()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1712_03439_gb300 import Plan, build, synth
    from paper_1712_03439_gb300 import _lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(v):
        return reduce_max(v, dist if world > 1 else None, dev)

    b = synth.config_home()
    audio_s = b.audio_seconds()
    plan = Plan.for_batch(b, eta_db=ETA_DB, gain_mode=0, device=dev.index,
                          spectrum_cache=not getattr(args, "no_spectrum_cache", False))
    x = torch.from_numpy(b.x).to(dev)
    rir = torch.from_numpy(b.rir).to(dev)
    snr = torch.from_numpy(b.snr_db).to(dev)
    gy = torch.from_numpy(synth.grad_like(99, b.y_size)).to(dev)
    gains = torch.empty(plan.S, device=dev)
    y = torch.empty(plan.y_size, device=dev)
    gx = torch.empty_like(x)
    gr = torch.empty_like(rir)
    gg = torch.empty_like(gains)
    tl = torch.empty(plan.R, dtype=torch.int32, device=dev)

    def fwd():
        plan.filter_mix(x, rir, gains, y, snr_db=snr, trunc_len=tl)

    def step():
        fwd()
        plan.filter_mix_backward(gy, x, gains, gx, gr, gg)

    for _ in range(max(args.warmup, 3)):
        step()
    plan.sync_status()
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    clock = ClockSampler(dev.index) if rank == 0 else None
    # ---- timed: K full steps (each call replays the plan's CUDA graphs)
    barrier()
    torch.cuda.synchronize()
    # an event between consecutive replays (outside the graphs) gives per-step times too
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    for k in range(args.steps):
        step()
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(evs[0].elapsed_time(evs[-1]) / args.steps)
    ms_median = max_over_ranks(float(np.median([evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)])))
    # ---- the same K steps with CUDA events around every stage (eager
    # launches: events inside a replayed graph cannot be read per step)
    plan.set_timing(True)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(args.steps):
        step()
    s1.record(stream)
    torch.cuda.synchronize()
    ms_eager = max_over_ranks(s0.elapsed_time(s1) / args.steps)
    stages = plan.stage_times()
    plan.set_timing(False)
    clocks = clock.stop() if clock else None
    plan.sync_status()

    if args.only_step:
        args.no_plain = args.no_cpu_baseline = True
    # ---- forward only (context)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kf = 0 if args.only_step else max(1, args.steps)
    barrier()
    f0.record(stream)
    for _ in range(kf):
        fwd()
    f1.record(stream)
    torch.cuda.synchronize()
    ms_fwd = max_over_ranks(f0.elapsed_time(f1) / kf) if kf else float("nan")

    # ---- end to end through the public API with host buffers: every step copies its
    # inputs in from pinned host memory and its results out; three device buffer sets
    # let step k's copies overlap the compute of its neighbours (copy-in and copy-out
    # on their own streams, ordered against the compute with events)
    pin = lambda t: t.cpu().pin_memory()
    hx, hrir, hsnr, hgy = pin(x), pin(rir), pin(snr), pin(gy)
    hy, hgx, hgr, hgg, hgains = (torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
                                 for t in (y, gx, gr, gg, gains))
    h2d = 4 * (hx.numel() + hrir.numel() + hsnr.numel() + hgy.numel())
    d2h = 4 * (hy.numel() + hgx.numel() + hgr.numel() + hgg.numel() + hgains.numel())
    ke = 0 if args.only_step else max(4, min(args.steps, 20))
    sets = [dict(x=x, rir=rir, snr=snr, gy=gy, gains=gains, y=y, gx=gx, gr=gr, gg=gg)]
    if ke:
        sets += [{k: torch.empty_like(v) for k, v in sets[0].items()} for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in sets]
    ev_done = [torch.cuda.Event() for _ in sets]
    ev_out = [torch.cuda.Event() for _ in sets]

    def e2e_step(k):
        bsel = k % len(sets)
        S = sets[bsel]
        with torch.cuda.stream(s_in):
            if k >= len(sets):
                s_in.wait_event(ev_out[bsel])          # this set's last results are out
            S["x"].copy_(hx, non_blocking=True)
            S["rir"].copy_(hrir, non_blocking=True)
            S["snr"].copy_(hsnr, non_blocking=True)
            S["gy"].copy_(hgy, non_blocking=True)
            ev_in[bsel].record(s_in)
        stream.wait_event(ev_in[bsel])
        plan.filter_mix(S["x"], S["rir"], S["gains"], S["y"], snr_db=S["snr"], stream=stream)
        plan.filter_mix_backward(S["gy"], S["x"], S["gains"], S["gx"], S["gr"], S["gg"], stream=stream)
        ev_done[bsel].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_done[bsel])
            hy.copy_(S["y"], non_blocking=True)
            hgx.copy_(S["gx"], non_blocking=True)
            hgr.copy_(S["gr"], non_blocking=True)
            hgg.copy_(S["gg"], non_blocking=True)
            hgains.copy_(S["gains"], non_blocking=True)
            ev_out[bsel].record(s_out)

    if ke:
        for k in range(len(sets)):                     # capture each set's graphs untimed
            e2e_step(k)
    torch.cuda.synchronize()
    barrier()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    s_in.wait_stream(stream)                          # copies start after the first event
    for k in range(ke):
        e2e_step(k)
    for k in range(len(sets)):
        stream.wait_event(ev_out[k])                   # the last results are on the host
    g1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(g0.elapsed_time(g1) / ke) if ke else float("nan")

    # ---- plain per-utterance GPU path (same step, torch.fft)
    plain = None
    if not args.no_plain:
        xs, hs, snrs, gys = _plain_inputs(torch, dev, b, x=x, rir=rir, snr=snr, gy=gy)
        plain_step(torch, b, xs, hs, snrs, gys)
        torch.cuda.synchronize()
        kp = 2
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(kp):
            plain_step(torch, b, xs, hs, snrs, gys)
        p1.record(stream)
        torch.cuda.synchronize()
        ms_plain = max_over_ranks(p0.elapsed_time(p1) / kp)
        plain = {"value": world * audio_s / (ms_plain / 1e3), "unit": UNIT, "ms_per_step": ms_plain,
                 "what": "per-utterance Python loop of full-length torch.fft (cuFFT) convolution "
                         "(Eq. 4) with torch truncation and gains, forward + autograd backward"}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel (from the live stage events)
    q = plan.query()
    L = tl.cpu().numpy()
    work = algorithmic_work(b, q, L, cache=plan.spectrum_cache)
    hbm, sm_mhz_max, peak_kind = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    p_fp32 = sms * 128 * 2 * sm_mhz_max * 1e6 / 1e12
    per = {k: (v[0] / v[1] if v[1] else 0.0) for k, v in stages.items()}
    kern = "backward" if per["backward"] >= per["forward"] else "forward"
    kname = {"forward": "k_forward", "backward": "k_backward_tm"}[kern]
    src = {"forward": "rsim_forward.cu", "backward": "rsim_backward.cu"}[kern]
    klabel = {"forward": "k_forward<M>",
              "backward": "k_backward_tm<M> (N <= 8192) and k_backward<8192> (N = 16384)"}[kern]
    n_sizes = plan.num_fft_sizes          # one launch per allowed FFT size
    w = "fwd" if kern == "forward" else "bwd"
    roof = roofline_entry(work[f"{w}_flops"], work[f"{w}_bytes"], per[kern], p_fp32, hbm, peak_kind,
                          _traffic_for(kname))
    roof.update({"kernel": f"{klabel} ({src}), all FFT-size launches of one step",
                 "stage_ms": per[kern], "launches_per_step": n_sizes,
                 "algorithmic_flops_per_step": work[f"{w}_flops"],
                 "algorithmic_bytes_per_step": work[f"{w}_bytes"],
                 "frac_5NlogN": work[f"{w}_flops_5n"] / (per[kern] / 1e3) / 1e12 / p_fp32,
                 "frac_5NlogN_note": "same kernel, counting 5 N log2 N flops per real N-point "
                                     "transform (the complex-FFT count) instead of 2.5 N log2 N"})
    fwd_roof = roofline_entry(work["fwd_flops"], work["fwd_bytes"], per["forward"], p_fp32, hbm,
                              peak_kind, _traffic_for("k_forward"))

    # ---- CPU oracle baseline on a bounded sample (rank 0, N = 1)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        cores = oracle.max_threads()
        n_cpu = min(b.num_utts, max(16, cores))
        sub = b.subset(range(n_cpu))
        g = synth.grad_like(99, sub.y_size)
        t0 = time.perf_counter()
        oracle_sample_step(oracle, sub, g)
        dt = time.perf_counter() - t0
        cpu = {"value": sub.audio_seconds() / dt, "unit": UNIT, "cores": cores,
               "kind": "oracle", "nproc": os.cpu_count(), "cpu_model": host_cpu(),
               "sample": f"utterances 0-{n_cpu - 1} of the home-256 batch ({sub.audio_seconds():.1f} s of audio), "
                         f"forward + backward, FP64 direct convolution on {cores} threads, {dt:.1f} s wall"}

    # truncate, power, gains, plan, backward partition, spectra, forward, fix-up | backward, finalize
    kernels_per_step = (5 + 2 * n_sizes + 1) + (n_sizes + 1)
    line = {
        "metric": METRIC, "value": whole_job_rate(audio_s, world, ms), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "ms_per_step_median": ms_median,
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": DATA,
        "config": {"workload": WORKLOAD, "global_batch": b.num_utts * world,
                   "audio_seconds_per_step": audio_s * world,
                   "step": "forward (cut-off, gains, FFT-size plan, RIR spectra, OLA filter-and-mix, "
                           "fix-up) + backward (grad x, grad RIR, grad gains), replayed as CUDA graphs",
                   "spectrum_cache": plan.spectrum_cache,
                   "l2": "inputs larger than L2 (x is %.0f MB, grad_y %.0f MB)"
                         % (x.numel() * 4 / 1e6, gy.numel() * 4 / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "fft_sizes_chosen": {str(1 << int(m)): int(c) for m, c in
                                        zip(*np.unique(q["log2_n"], return_counts=True))}},
        "fwd_only": {"value": world * audio_s / (ms_fwd / 1e3), "unit": UNIT, "ms_per_step": ms_fwd,
                     "roofline": fwd_roof},
        "stages_ms_per_step": per,
        "eager_ms_per_step": ms_eager,
        "roofline": roof,
        "step_roofline": step_roofline(work, ms, p_fp32, hbm),
        "fp32_peak_cross_check": {"derived_tflops": p_fp32, "probe": probe_fp32(dev.index),
                                  "probe_what": "8 independent FMA chains per thread, full occupancy "
                                                "(paper_1712_03439_gb300/probe/fp32_peak.cu)"},
        "cpu_baseline": cpu,
        "plain_gpu": plain,
        "e2e": {"value": world * audio_s / (ms_e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e},
        "gpu_launches": kernels_per_step * args.steps,
        "clocks": clocks,
    }
    if plain:
        line["vs_plain"] = line["value"] / plain["value"]
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# other workloads (reports beside the headline; not the default line)
# ---------------------------------------------------------------------------
def probe_fp32(device=0):
    """FP32 FMA throughput measured by the probe kernel (TFLOP/s), or None."""
    import ctypes
    try:
        from paper_1712_03439_gb300 import build
        lib = ctypes.CDLL(build.build_probe())
    except (OSError, RuntimeError):
        return None
    tf, ms = ctypes.c_double(), ctypes.c_double()
    lib.fp32_peak_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    if lib.fp32_peak_probe(int(device), 4096, 5, ctypes.byref(tf), ctypes.byref(ms)) != 0:
        return None
    return {"tflops": tf.value, "ms": ms.value}


def _peaks_fp32(torch, dev):
    hbm, sm_mhz_max, peak_kind = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return hbm, sms * 128 * 2 * sm_mhz_max * 1e6 / 1e12, peak_kind


def run_stream(args):
    """Streaming queue of utterances (log-uniform 0.5-20 s, 1-4 sources, 2 mics)
    in device-resident batches admitted by a memory budget, forward + backward."""
    import torch
    from paper_1712_03439_gb300 import build, synth
    from paper_1712_03439_gb300.stream import Streamer
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    build.build()
    b = synth.config_stream(n_utts=args.stream_utts)
    st = Streamer(budget_bytes=int(args.budget_gb * (1 << 30)), eta_db=ETA_DB, backward=True,
                  keep_outputs=False, class_plan=not args.stream_plan_per_batch)
    st.run(b.subset(range(min(64, b.num_utts))))          # warm-up (context, code, allocator)
    clock = ClockSampler(0)
    t0 = time.perf_counter()
    res = st.run(b)
    wall = time.perf_counter() - t0
    clocks = clock.stop()
    hbm, p_fp32, peak_kind = _peaks_fp32(torch, dev)
    flops = nbytes = 0.0
    off = 0
    for r in res.records:
        sub = b.subset(r.utts)
        w = algorithmic_work(sub, r.query, r.trunc_len)
        flops += w["fwd_flops"] + w["bwd_flops"]
        nbytes += w["fwd_bytes"] + w["bwd_bytes"]
    dev_s = sum(r.device_ms for r in res.records) / 1e3
    t_roof = max(nbytes / (hbm * 1e9), flops / (p_fp32 * 1e12))
    plain = None
    if not args.no_plain:
        sub = b.subset(range(min(64, b.num_utts)))
        plain = _plain_rate(torch, dev, sub)
    wall_sum = sum(r.wall_ms for r in res.records) / 1e3
    line = {"metric": "simulated audio s/sec (fwd+bwd), streaming batches admitted by memory budget",
            "value": res.audio_seconds / wall_sum, "unit": UNIT,
            "value_note": "audio seconds / sum of per-batch wall latencies (batches run one after "
                          "another); the harness's own host work (forming batches, synthetic "
                          f"gradients) is outside, {wall:.1f} s in all", "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32", "data": DATA,
            "config": {"workload": f"stream-{b.num_utts}: lengths log-uniform 0.5-20 s, 1-4 sources, "
                                   f"2 mics, RT60 U(0.1,0.9) s, eta {ETA_DB:g} dB",
                       "budget_gb": args.budget_gb, "batches": len(res.records),
                       "audio_seconds": res.audio_seconds},
            "value_device": res.audio_seconds / dev_s,
            "latency_ms": {"p50_wall": res.latency_ms(50), "p99_wall": res.latency_ms(99),
                           "p50_device": res.latency_ms(50, "device_ms"),
                           "p99_device": res.latency_ms(99, "device_ms"),
                           "p50_plan": res.latency_ms(50, "plan_ms"),
                           "p50_staging": res.latency_ms(50, "staging_ms")},
            "batches_on_the_shape_class_plan": int(sum(r.reshaped for r in res.records)),
            "note": "wall: batch inputs in pinned host memory to results on the host (re-planning the "
                    "shape-class plan, copies both ways, kernels); staging: the host copy of a batch's "
                    "inputs into pinned memory, done on a host thread while the previous batch runs; "
                    "device: first copy to last copy on the stream",
            "roofline": {"t_roof_s": t_roof, "device_s": dev_s, "frac": t_roof / dev_s,
                         "bound": "alu" if flops / (p_fp32 * 1e12) >= nbytes / (hbm * 1e9) else "hbm",
                         "peak_fp32_tflops": p_fp32, "peak_hbm_gbs": hbm, "peak_source": peak_kind},
            "max_footprint_gb": max(r.footprint_bytes for r in res.records) / (1 << 30),
            "plain_gpu": plain, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def _plain_rate(torch, dev, sub):
    xs, hs, snrs, gys = _plain_inputs(torch, dev, sub)
    plain_step(torch, sub, xs, hs, snrs, gys)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_step(torch, sub, xs, hs, snrs, gys)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"value": sub.audio_seconds() / dt, "unit": UNIT, "sample": f"{sub.num_utts} utterances"}


def run_long(args):
    """Long reverberant multi-mic workload (30 s, 4 sources, 8 mics, RT60 0.8-1.2 s):
    cut-off sweep with work saved, energy error and forward+backward throughput."""
    import torch
    from paper_1712_03439_gb300 import Plan, build, synth
    from paper_1712_03439_gb300._lib import RsimError
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    build.build()
    b = synth.config_long(n_utts=args.long_utts)
    audio_s = b.audio_seconds()
    x, rir = torch.from_numpy(b.x).to(dev), torch.from_numpy(b.rir).to(dev)
    snr = torch.from_numpy(b.snr_db).to(dev)
    gy = torch.from_numpy(synth.grad_like(98, b.y_size)).to(dev)
    # reference without a cut-off (full-length FFT convolution with torch.fft, FP64) on
    # two utterances, for the output error each cut-off costs
    ref_utts = [0, 1] if b.num_utts > 1 else [0]
    si, xo, yo, ri, ro = b.src_index(), b.x_offsets(), b.y_offsets(), b.rir_index(), b.rir_offsets()
    rhat = {}
    for u in ref_utts:
        I, nx, J = int(b.num_sources[u]), int(b.num_samples[u]), b.num_mics
        xs = torch.from_numpy(b.x[xo[si[u]]:xo[si[u + 1]]].reshape(I, nx)).to(dev, torch.float64)
        hs = [torch.from_numpy(b.rir[ro[r]:ro[r + 1]]).to(dev, torch.float64) for r in range(ri[u], ri[u + 1])]
        n = 1 << int(math.ceil(math.log2(nx + max(h.numel() for h in hs) - 1)))
        X = torch.fft.rfft(xs, n)
        rhat[u] = (X, hs, n)
    sweep = []
    clock = ClockSampler(0)
    for eta in (10.0, 20.0, 30.0, math.inf):
        ent = {"eta_db": None if math.isinf(eta) else eta}
        plan = Plan.for_batch(b, eta_db=eta, gain_mode=0, device=0)
        gains, y = torch.empty(plan.S, device=dev), torch.empty(plan.y_size, device=dev)
        tl = torch.empty(plan.R, dtype=torch.int32, device=dev)
        ek = torch.empty(plan.R, device=dev)
        gx, gr, gg = torch.empty_like(x), torch.empty_like(rir), torch.empty_like(gains)

        def step():
            plan.filter_mix(x, rir, gains, y, snr_db=snr, trunc_len=tl, energy_kept_frac=ek)
            plan.filter_mix_backward(gy, x, gains, gx, gr, gg)
        try:
            step()
            plan.sync_status()
        except RsimError as e:
            L = oracle_free_lengths(b, eta)
            ent.update(unsupported=str(e), longest_kept_rir=int(L.max()),
                       work_saved=float(np.sum(b.rir_len - L) / np.sum(b.rir_len)))
            sweep.append(ent)
            plan.close()
            continue
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.long_steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.long_steps
        L = tl.cpu().numpy().astype(np.int64)
        a = gains.cpu().numpy().astype(np.float64)
        errs = []
        for u in ref_utts:
            X, hs, n = rhat[u]
            I, nx, J = int(b.num_sources[u]), int(b.num_samples[u]), b.num_mics
            H = torch.stack([torch.fft.rfft(h, n) for h in hs]).reshape(I, J, -1)
            A = torch.from_numpy(a[si[u]:si[u + 1]]).to(dev)
            yref = torch.fft.irfft(torch.einsum("i,if,ijf->jf", A.to(X.dtype), X, H), n)[:, :nx]
            yg = y[yo[u]:yo[u + 1]].reshape(J, nx).to(torch.float64)
            errs.append(float(torch.linalg.norm(yg - yref) / torch.linalg.norm(yref)))
        q = plan.query()
        ent.update(value=audio_s / (ms / 1e3), unit=UNIT, ms_per_step=ms,
                   work_saved=float(np.sum(b.rir_len - L) / np.sum(b.rir_len)),
                   mean_kept_taps=float(L.mean()), longest_kept_rir=int(L.max()),
                   energy_kept_frac_mean=float(ek.mean().item()),
                   output_rel_l2_vs_no_cutoff=float(np.mean(errs)),
                   fft_sizes={int(k): int(c) for k, c in zip(*np.unique(1 << q["log2_n"].astype(np.int64),
                                                                        return_counts=True))})
        sweep.append(ent)
        plan.close()
    clocks = clock.stop()
    line = {"metric": "simulated audio s/sec (fwd+bwd) per cut-off, long reverberant multi-mic",
            "unit": UNIT, "n_gpus": 1, "dtype": "f32", "data": DATA, "higher_is_better": True,
            "config": {"workload": f"long-{b.num_utts}: {b.num_utts} x 30 s, 4 sources, 8-mic circle r=5 cm, "
                                   "RT60 U(0.8,1.2) s", "audio_seconds": audio_s,
                       "energy_error_reference": "full-length torch.fft FP64 convolution without cut-off, "
                                                 f"utterances {ref_utts}"},
            "sweep": sweep, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def image_work(geom_rows: int, rir_len, order: int):
    """Algorithmic work of rsim_image_rirs: every tap written once (zeros
    included) and each RIR's 40-byte geometry and 8-byte offset read; per
    image one FP32 add pair, square root, multiply and two divisions (counted
    as 6 flops), for the (2K+1)^3 images of every RIR."""
    taps = int(np.sum(np.asarray(rir_len, dtype=np.int64)))
    nbytes = 4.0 * taps + 48.0 * geom_rows + 8.0
    flops = 6.0 * geom_rows * (2 * order + 1) ** 3
    return nbytes, flops


def run_rooms(args):
    """Image-method RIRs (Eq. 1, 17^3 virtual rooms) for the Home mix, made on
    the device and fed to the filter-and-mix step: the generator's own time and
    roofline, and the whole step (RIRs + forward + backward)."""
    import torch
    from paper_1712_03439_gb300 import Plan, build, image_rirs, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    build.build()
    order = 8
    b, geom = synth.config_home_rooms()
    lens = b.rir_len.astype(np.int64)
    off = np.concatenate([[0], np.cumsum(lens)])
    audio_s = b.audio_seconds()
    g_d, off_d = torch.from_numpy(geom).to(dev), torch.from_numpy(off).to(dev)
    rir = torch.empty(int(off[-1]), device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    x, snr = torch.from_numpy(b.x).to(dev), torch.from_numpy(b.snr_db).to(dev)
    gy = torch.from_numpy(synth.grad_like(97, b.y_size)).to(dev)
    hbm, p_fp32, peak_kind = _peaks_fp32(torch, dev)
    # the generator alone: its 41 MB output fits in L2, so L2 is flushed (a 256 MB
    # write) before every timed launch and each launch is timed on its own
    flush = torch.empty(64 << 20, device=dev)
    st = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        image_rirs(g_d, off_d, int(lens.max()), rir, order=order, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0, "invalid room geometry"
    n_img = max(args.steps, 20)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_img)]
    clock = ClockSampler(0)
    for e0, e1 in evs:
        flush.fill_(1.0)
        e0.record(st)
        image_rirs(g_d, off_d, int(lens.max()), rir, order=order)
        e1.record(st)
    torch.cuda.synchronize()
    img_ms = float(np.mean([a.elapsed_time(z) for a, z in evs]))
    nbytes, flops = image_work(geom.shape[0], lens, order)
    img_roof = roofline_entry(flops, nbytes, img_ms, p_fp32, hbm, peak_kind, _traffic_for("k_image_rirs"))
    # the step: RIRs from the rooms, then forward and backward
    plan = Plan.for_batch(b, eta_db=ETA_DB, gain_mode=0, device=0)
    gains, y = torch.empty(plan.S, device=dev), torch.empty(plan.y_size, device=dev)
    gx, gr, gg = torch.empty_like(x), torch.empty_like(rir), torch.empty_like(gains)

    def step():
        image_rirs(g_d, off_d, int(lens.max()), rir, order=order)
        plan.filter_mix(x, rir, gains, y, snr_db=snr)
        plan.filter_mix_backward(gy, x, gains, gx, gr, gg)
    for _ in range(max(args.warmup, 3)):
        step()
    plan.sync_status()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    q = plan.query()
    plan.close()
    # the fused step: RIRs made where they are consumed (generation and cut-off in one
    # kernel, only the kept taps written), then forward and backward
    fplan = Plan.for_batch(b, eta_db=ETA_DB, gain_mode=0, device=0, rooms=True)
    fgains, fy = torch.empty(fplan.S, device=dev), torch.empty(fplan.y_size, device=dev)
    fgx, fgr, fgg = torch.empty_like(x), torch.empty_like(rir), torch.empty_like(fgains)

    def fused_step():
        fplan.filter_mix_rooms(x, g_d, fgains, fy, snr_db=snr, order=order)
        fplan.filter_mix_backward(gy, x, fgains, fgx, fgr, fgg)
    for _ in range(max(args.warmup, 3)):
        fused_step()
    fplan.sync_status()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(args.steps):
        fused_step()
    e1.record(st)
    torch.cuda.synchronize()
    fms = e0.elapsed_time(e1) / args.steps
    fplan.close()
    clocks = clock.stop()
    line = {"metric": "simulated audio s/sec (image-method RIRs + fwd + bwd) at 16 kHz, 1xGB300",
            "value": audio_s / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic: the Home mix's signals with image-method rooms (seeded)",
            "config": {"workload": f"home-rooms-{b.num_utts}: the Home mix, one cuboid room per utterance "
                                   "(3-10 x 3-8 x 2.5-5 m, Sabine reflection from RT60 U(0.1,0.9) s), "
                                   f"{geom.shape[0]} RIRs of ceil(RT60 fs) taps, {(2 * order + 1) ** 3} "
                                   "virtual rooms each, eta 20 dB",
                       "audio_seconds": audio_s, "rirs": int(geom.shape[0]), "taps": int(off[-1]),
                       "fft_sizes": {int(k): int(c) for k, c in zip(*np.unique(
                           1 << q["log2_n"].astype(np.int64), return_counts=True))},
                       "l2": "generator timed alone after a 256 MB L2 flush per launch; the step's "
                             "inputs (x 0.35 GB) are larger than L2"},
            "image_rirs": {"ms": img_ms, "launches_timed": n_img, "rirs_per_s": geom.shape[0] / (img_ms / 1e3),
                           "roofline": img_roof},
            "fused": {"value": audio_s / (fms / 1e3), "unit": UNIT, "ms_per_step": fms,
                      "what": "rsim_filter_mix_rooms: each RIR's images land in shared memory, the cut-off "
                              "is taken there and only the kept taps are written; then the spectra, "
                              "forward and backward (the headline value above is the two-call step: "
                              "rsim_image_rirs writes every tap, rsim_filter_mix reads them)"},
            "clocks": clocks}
    if not args.no_cpu_baseline:
        import oracle
        oracle.image_rirs(geom[:8], lens[:8], order=order)     # builds and loads the oracle
        t0 = time.perf_counter()
        oracle.image_rirs(geom, lens, order=order)
        cpu_s = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": geom.shape[0] / cpu_s, "unit": "RIRs/s", "cores": oracle.max_threads(),
                                "kind": "oracle",
                                "sample": f"all {geom.shape[0]} RIRs of the workload (FP64 amplitudes)"}
    print(json.dumps(line), flush=True)
    return 0


def mel_work(num_out, rows_total, frames_total, n_mels=128, stack=4):
    """Algorithmic work of rsim_plan_log_mel: the channel read once (4 bytes a
    sample) and the features written once; per frame the window (512
    multiplies), one real 512-point transform (2.5 N log2 N), the power
    spectrum (3 per bin) and the filter sums (2 per weighted bin, about two
    filters per bin)."""
    nbytes = 4.0 * float(np.sum(num_out)) + 4.0 * rows_total * stack * n_mels
    flops = frames_total * (512 + 2.5 * 512 * 9 + 3 * 257 + 2 * 2 * 257)
    return nbytes, flops


def run_mel(args):
    """Log-Mel front end (Sec. 3: 128 filters, 32 ms / 10 ms, 125-7500 Hz, four
    frames stacked, every third kept) on microphone 0 of the home-256 mix."""
    import torch
    from paper_1712_03439_gb300 import Plan, build, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    build.build()
    b = synth.config_home()
    plan = Plan.for_batch(b, eta_db=ETA_DB, gain_mode=0, device=0)
    x, rir, snr = (torch.from_numpy(a).to(dev) for a in (b.x, b.rir, b.snr_db))
    gains, y = torch.empty(plan.S, device=dev), torch.empty(plan.y_size, device=dev)
    plan.filter_mix(x, rir, gains, y, snr_db=snr)
    rows, total = plan.log_mel_rows()
    feats = torch.empty((total, 512), device=dev)
    frames = int(np.sum(np.where(rows > 0, (rows - 1) * 3 + 4, 0)))
    flush = torch.empty(64 << 20, device=dev)
    st = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        plan.log_mel(y, feats)
    torch.cuda.synchronize()
    n = max(args.steps, 20)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    clock = ClockSampler(0)
    for e0, e1 in evs:
        flush.fill_(1.0)
        e0.record(st)
        plan.log_mel(y, feats)
        e1.record(st)
    torch.cuda.synchronize()
    clocks = clock.stop()
    ms = float(np.mean([a.elapsed_time(z) for a, z in evs]))
    hbm, p_fp32, peak_kind = _peaks_fp32(torch, dev)
    nbytes, flops = mel_work(plan.num_out, total, frames)
    audio_s = b.audio_seconds()
    line = {"metric": "log-Mel features of the mixed output, audio s/sec (1 channel) at 16 kHz, 1xGB300",
            "value": audio_s / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": n, "warmup": max(args.warmup, 3),
            "ms_per_step": ms, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic: microphone 0 of the home-256 mix (filter_mix output)",
            "config": {"workload": "home-256 mixed output, microphone 0: 128 log-Mel filters over 125-7500 Hz, "
                                   "512-sample Hann frames every 160 samples, 4 frames stacked, every third kept",
                       "audio_seconds": audio_s, "frames": frames, "rows": total,
                       "l2": "each timed launch follows a 256 MB L2 flush"},
            "roofline": roofline_entry(flops, nbytes, ms, p_fp32, hbm, peak_kind, _traffic_for("k_log_mel")),
            "clocks": clocks}
    if not args.no_cpu_baseline:
        import oracle
        sub = list(range(0, b.num_utts, 64))[:4]
        yo, yh = b.y_offsets(), y.cpu().numpy()
        t0 = time.perf_counter()
        sec = 0.0
        for u in sub:
            nu = int(b.num_samples[u])
            oracle.log_mel(yh[yo[u]:yo[u] + nu])
            sec += nu / synth.FS
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": sec / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"utterances {sub} ({sec:.1f} audio s), one thread"}
    plan.close()
    print(json.dumps(line), flush=True)
    return 0


def run_gains(args):
    """Forward + backward on the home-256 mix under each gain mode: 0 (SNRs on the
    dry signals), 2 (one gain per source and microphone) and 3 (SNRs on the
    reverberant signal at microphone 0, one more filtering pass per source)."""
    import torch
    from paper_1712_03439_gb300 import Plan, build, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    build.build()
    b = synth.config_home()
    audio_s = b.audio_seconds()
    x, rir, snr = (torch.from_numpy(a).to(dev) for a in (b.x, b.rir, b.snr_db))
    gy = torch.from_numpy(synth.grad_like(95, b.y_size)).to(dev)
    steps = max(args.steps // 10, 10)
    out = {}
    clock = ClockSampler(0)
    for mode in (0, 2, 3):
        plan = Plan.for_batch(b, eta_db=ETA_DB, gain_mode=mode, device=0)
        gains = (torch.from_numpy(np.repeat(np.linspace(0.5, 1.0, plan.S), b.num_mics).astype(np.float32)).to(dev)
                 if mode == 2 else torch.empty(plan.G, device=dev))
        y = torch.empty(plan.y_size, device=dev)
        gx, gr, gg = torch.empty_like(x), torch.empty_like(rir), torch.empty(plan.G, device=dev)

        def step():
            plan.filter_mix(x, rir, gains, y, snr_db=None if mode == 2 else snr)
            plan.filter_mix_backward(gy, x, gains, gx, gr, gg)
        for _ in range(3):
            step()
        plan.sync_status()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[str(mode)] = {"ms_per_step": ms, "value": audio_s / (ms / 1e3), "unit": UNIT}
        plan.close()
    line = {"metric": "simulated audio s/sec (fwd+bwd) per gain mode, home-256", "unit": UNIT, "n_gpus": 1,
            "dtype": "f32", "data": DATA, "higher_is_better": True, "steps": steps,
            "config": {"workload": WORKLOAD, "gain_modes": {"0": "SNRs on the dry signals",
                                                             "2": "one gain per source and microphone",
                                                             "3": "SNRs on the reverberant signal at mic 0"}},
            "modes": out, "clocks": clock.stop()}
    print(json.dumps(line), flush=True)
    return 0


def oracle_free_lengths(b, eta):
    """Kept lengths (Eq. 7-9) computed in numpy for the report when the library
    rejects the batch (FP64 compare, as the kernels do)."""
    ro = b.rir_offsets()
    out = np.zeros(b.num_rirs, np.int64)
    fac = 0.0 if math.isinf(eta) else 10.0 ** (-eta / 10.0)
    for r in range(b.num_rirs):
        h2 = b.rir[ro[r]:ro[r + 1]].astype(np.float64) ** 2
        if math.isinf(eta) or h2.max() == 0:
            out[r] = h2.size if math.isinf(eta) else 1
            continue
        idx = np.nonzero(h2 >= h2.max() * fac)[0]
        out[r] = min(int(idx[-1]) + 2, h2.size)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-spectrum-cache", action="store_true",
                    help="home workload: the backward transforms every source block again instead of "
                         "reading the forward's spectra")
    ap.add_argument("--only-step", action="store_true",
                    help="time only the K steps (no forward-only, end-to-end, plain or CPU legs); "
                         "for profiler runs")
    ap.add_argument("--config", choices=["home", "stream", "long", "rooms", "mel", "gains"], default="home",
                    help="home: the headline line; stream / long / rooms / mel: reports on the streaming, "
                         "the long reverberant and the image-method-room workloads and on the log-Mel "
                         "front end")
    ap.add_argument("--stream-utts", type=int, default=4096)
    ap.add_argument("--budget-gb", type=float, default=2.0)
    ap.add_argument("--stream-plan-per-batch", action="store_true",
                    help="stream: a plan made for every batch instead of one re-planned shape-class plan")
    ap.add_argument("--long-utts", type=int, default=32)
    ap.add_argument("--long-steps", type=int, default=5)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "stream":
        return run_stream(args)
    if args.config == "long":
        return run_long(args)
    if args.config == "rooms":
        return run_rooms(args)
    if args.config == "mel":
        return run_mel(args)
    if args.config == "gains":
        return run_gains(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
