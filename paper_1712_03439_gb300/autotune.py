"""Autotuner for the FFT-size choice and the work-tile lengths.

The planner picks, per utterance, the FFT size N minimising
(blocks(N) * (I + J) + I * J) * cost[N] (Eq. 6's structure with measured
per-size costs).  This module measures cost[N] on the device: for each
allowed N it runs the forward and backward on a workload where every size is
admissible, reads the kernels' CUDA-event stage times and divides by the
number of block transforms.  It then times the benchmark-shaped workload for
a few forward tile lengths.  The result is stored as JSON keyed by
the GPU name in ``tuning.json`` next to this file; ``Plan`` loads it when no
cost table is given.

  python -m paper_1712_03439_gb300.autotune [--out PATH]
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")
SIZES = (2048, 4096, 8192, 16384)


def load_table(gpu_name: str):
    if not os.path.exists(TABLE):
        return None
    return json.load(open(TABLE)).get(gpu_name)


def _time_plan(plan, x, rir, gains, y, gy, gx, gr, gg, reps):
    import torch
    for _ in range(3):
        plan.filter_mix(x, rir, gains, y)
        plan.filter_mix_backward(gy, x, gains, gx, gr, gg)
    plan.sync_status()
    plan.set_timing(True)
    for _ in range(reps):
        plan.filter_mix(x, rir, gains, y)
        plan.filter_mix_backward(gy, x, gains, gx, gr, gg)
    st = plan.stage_times()
    plan.set_timing(False)
    torch.cuda.synchronize()
    return {k: v[0] / max(v[1], 1) for k, v in st.items()}


def _buffers(b, dev):
    import torch
    from . import synth
    x = torch.from_numpy(b.x).to(dev)
    rir = torch.from_numpy(b.rir).to(dev)
    S = int(b.num_sources.sum())
    gains = torch.linspace(0.5, 1.0, S, device=dev)
    y = torch.empty(b.y_size, device=dev)
    gy = torch.from_numpy(synth.grad_like(3, b.y_size)).to(dev)
    return x, rir, gains, y, gy, torch.empty_like(x), torch.empty_like(rir), torch.empty_like(gains)


def measure_fft_costs(device=0, sizes=SIZES, reps=5):
    """ns per (block x (sources + mics)) of forward + backward, per FFT size."""
    import torch
    from . import synth
    from .api import Plan
    dev = torch.device("cuda", device)
    # short reverberation: every size admits the truncated RIRs (L <= 1025)
    rng = np.random.Generator(np.random.PCG64(5))
    n = 48
    lengths = (rng.uniform(4.0, 12.0, n) * synth.FS).astype(np.int64)
    n_src = 1 + rng.integers(0, 4, n)
    b = synth.make_batch(171203439 + 50, lengths, n_src, synth.linear_pair_array(), (0.05, 0.1))
    bufs = _buffers(b, dev)
    out = {}
    for N in sizes:
        plan = Plan.for_batch(b, eta_db=20.0, fft_sizes=[N], gain_mode=1, device=device)
        t = _time_plan(plan, *bufs, reps)
        q = plan.query()
        units = float(np.sum(q["num_blocks"] * (b.num_sources + b.num_mics)))
        out[N] = 1e6 * (t["forward"] + t["backward"] + t["spectrum"]) / units
        plan.close()
    return out


def measure_tiles(costs, device=0, reps=5):
    """Best forward segment length on the Home-like workload (the backward is
    partitioned on the device, one equal-cost chunk per CTA)."""
    import torch
    from . import synth
    from .api import Plan
    dev = torch.device("cuda", device)
    b = synth.config_home(n_utts=128)
    bufs = _buffers(b, dev)
    best = None
    for fseg in (16384, 32768, 65536):
        plan = Plan.for_batch(b, eta_db=20.0, gain_mode=1, segment_len=fseg, fft_cost=costs, device=device)
        t = _time_plan(plan, *bufs, reps)
        plan.close()
        if best is None or t["forward"] < best[0]:
            best = (t["forward"], fseg)
    return {"segment_len": best[1]}


def autotune(device=0, out=TABLE):
    import torch
    name = torch.cuda.get_device_name(device)
    costs = measure_fft_costs(device)
    tiles = measure_tiles(costs, device)
    entry = {"fft_cost_ns": {str(k): v for k, v in costs.items()}, **tiles}
    table = json.load(open(out)) if os.path.exists(out) else {}
    table[name] = entry
    with open(out, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    return name, entry


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--device", type=int, default=0)
    a = ap.parse_args()
    print(json.dumps(autotune(a.device, a.out)))
