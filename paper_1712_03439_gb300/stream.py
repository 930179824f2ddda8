"""Streaming execution: a queue of utterances processed in device-resident
batches admitted by a memory budget.

Utterances are taken in queue order; a batch grows while its device footprint
(inputs, outputs, gradients and the plan's scratch) stays within the budget.
Each batch is copied to the device from pinned staging buffers, planned, run
forward (and backward with a given upstream gradient), and its results are
copied back.  Per batch the host wall time from admission to results on the
host, and the device time between its first copy and its last, are recorded.

The footprint estimate follows the plan's scratch layout (RIR spectra at the
largest allowed FFT size, per-segment carries, the backward partition and its
RIR-gradient partials); after the plan is made its real scratch size replaces
the estimate in the record.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

from . import synth

_MAX_LOG = 14                      # largest FFT size the kernels support (2^14)
_MMAX = 1 << (_MAX_LOG - 1)
_POWER_CHUNK = 32768
# per-plan bytes that do not grow with the batch: twiddle tables of every FFT size
# (two thread shapes each), queue cursors, error words and the 256-byte alignment of
# about thirty pieces
PLAN_FIXED_BYTES = 2 << 20


# CTAs of the backward launches of all FFT sizes together (the partition allots
# one chunk to each): SMs x (2 + 2 + 1 + 1) on a 152-SM GB300
PART_CTAS = 152 * 6


def utterance_bytes(nx: int, n_src: int, n_mics: int, rir_sum: int, nh_max: int, *,
                    backward: bool = True, output_mode: int = 0, seg_len: int = 16384) -> int:
    """Device bytes one utterance adds to a batch: its buffers plus its share of
    the plan's scratch (an estimate of the library's allocation; the backward
    partition's per-CTA share is in partition_bytes)."""
    ny = nx + (nh_max - 1 if output_mode else 0)
    buf = 4 * (n_src * nx + rir_sum + n_mics * ny) + 8 * n_src
    if backward:
        buf += 4 * (n_mics * ny + n_src * nx + rir_sum) + 4 * n_src
    nseg = -(-nx // max(seg_len, 1 << _MAX_LOG))
    scratch = 8 * n_src * n_mics * _MMAX                 # RIR spectra
    scratch += 4 * nseg * n_mics * 2 * _MMAX             # segment carries
    scratch += 4 * rir_sum                               # RIR-gradient partials (one piece per stream)
    scratch += 8 * n_src * (-(-nx // _POWER_CHUNK))      # power partial sums
    scratch += 4 * 3 * 4 * max(nseg, n_src * n_mics) + 256
    # backward streams: order and cost prefix per size, first and last piece, one piece
    # with its partial offset and source-gain partials
    scratch += n_src * (4 * 4 + 8 * 4 + 4 + 4 + 8 + 4 * 16)
    return int(buf + scratch)


def partition_bytes(utt_taps_max: int, ctas: int = PART_CTAS) -> int:
    """The backward partition's per-CTA scratch: one extra piece per CTA boundary
    (partial offset, source-gain partials, RIR-gradient partials of up to the
    largest utterance's taps) and the chunk starts."""
    return int(ctas * (8 + 4 * 16 + 4 * utt_taps_max + 3 * 4))


def group_bytes(batch: synth.Batch, utts, **kw) -> int:
    """Estimated device footprint of a batch made of the given utterances."""
    ri = batch.rir_index()
    total, taps_max = PLAN_FIXED_BYTES, 0
    for u in utts:
        lens = batch.rir_len[ri[u]:ri[u + 1]]
        total += utterance_bytes(int(batch.num_samples[u]), int(batch.num_sources[u]), batch.num_mics,
                                 int(lens.sum()), int(lens.max()), **kw)
        taps_max = max(taps_max, int(lens.sum()))
    return int(total + partition_bytes(taps_max))


def admit(batch: synth.Batch, budget_bytes: int, **kw) -> list[range]:
    """Consecutive groups of utterances whose estimated footprint fits the budget
    (an utterance larger than the budget forms a group of its own)."""
    ri = batch.rir_index()
    groups, start, used, taps_max = [], 0, PLAN_FIXED_BYTES, 0
    for u in range(batch.num_utts):
        lens = batch.rir_len[ri[u]:ri[u + 1]]
        b = utterance_bytes(int(batch.num_samples[u]), int(batch.num_sources[u]), batch.num_mics,
                            int(lens.sum()), int(lens.max()), **kw)
        taps = int(lens.sum())
        if u > start and used + b + partition_bytes(max(taps_max, taps)) > budget_bytes:
            groups.append(range(start, u))
            start, used, taps_max = u, PLAN_FIXED_BYTES, 0
        used += b
        taps_max = max(taps_max, taps)
    if start < batch.num_utts:
        groups.append(range(start, batch.num_utts))
    return groups


@dataclasses.dataclass
class BatchRecord:
    utts: range
    audio_seconds: float
    wall_ms: float          # inputs formed on the host to results on the host
    device_ms: float        # first host-to-device copy to last device-to-host copy
    plan_ms: float          # making the plan (allocation and table upload)
    footprint_bytes: int    # buffers + the plan's real scratch
    fft_blocks: dict        # FFT size -> utterances that used it
    query: dict             # the plan's per-utterance choice (log2 N, hop, L_max, blocks)
    trunc_len: np.ndarray   # kept RIR lengths of the batch


@dataclasses.dataclass
class StreamResult:
    records: list
    outputs: list           # per batch: dict of host arrays (y, gains, trunc_len, grads)

    @property
    def audio_seconds(self) -> float:
        return float(sum(r.audio_seconds for r in self.records))

    def latency_ms(self, q: float, kind: str = "wall_ms") -> float:
        v = np.array([getattr(r, kind) for r in self.records])
        return float(np.percentile(v, q)) if v.size else math.nan


class Streamer:
    """Runs a queue of utterances through the library in budget-sized batches."""

    def __init__(self, budget_bytes: int = 8 << 30, eta_db: float = 20.0, backward: bool = True,
                 output_mode: int = 0, device=None, keep_outputs: bool = True, **plan_kw):
        import torch
        self.torch = torch
        self.budget = int(budget_bytes)
        self.eta_db = float(eta_db)
        self.backward = bool(backward)
        self.output_mode = int(output_mode)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.keep = keep_outputs
        # one call per plan: launch eagerly rather than capture a graph that is never replayed
        self.plan_kw = dict(graphs=False, **plan_kw)
        self._pin = {}

    def _staging(self, name, n, dtype):
        t = self._pin.get(name)
        if t is None or t.numel() < n or t.dtype != dtype:
            t = self.torch.empty(max(n, 1), dtype=dtype, pin_memory=True)
            self._pin[name] = t
        return t[:n]

    def run(self, batch: synth.Batch, grad_y=None, groups=None) -> StreamResult:
        """grad_y(sub_batch, ny) -> float32 upstream gradient for a batch (or None:
        a seeded one).  Returns per-batch records and (if kept) outputs."""
        torch = self.torch
        from .api import Plan
        dev = self.device
        stream = torch.cuda.current_stream(dev)
        groups = groups if groups is not None else admit(batch, self.budget, backward=self.backward,
                                                         output_mode=self.output_mode)
        records, outputs = [], []
        for gi, grp in enumerate(groups):
            sub = batch.subset(grp)
            ny = synth.output_lengths(sub, self.output_mode)
            gy = (grad_y(sub, ny) if grad_y is not None
                  else synth.grad_like(1000 + gi, int(ny.sum()) * sub.num_mics)) if self.backward else None
            # the batch's latency runs from here: inputs formed on the host
            t0 = time.perf_counter()
            # pinned staging, then asynchronous copies on the current stream
            hx = self._staging("x", sub.x.size, torch.float32)
            hr = self._staging("rir", sub.rir.size, torch.float32)
            hs = self._staging("snr", sub.snr_db.size, torch.float32)
            hx.numpy()[:] = sub.x
            hr.numpy()[:] = sub.rir
            hs.numpy()[:] = sub.snr_db
            if gy is not None:
                hg = self._staging("gy", gy.size, torch.float32)
                hg.numpy()[:] = gy
            tp = time.perf_counter()
            plan = Plan.for_batch(sub, eta_db=self.eta_db, output_mode=self.output_mode, device=dev.index,
                                  **self.plan_kw)
            plan_ms = (time.perf_counter() - tp) * 1e3
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x = hx.to(dev, non_blocking=True)
            rir = hr.to(dev, non_blocking=True)
            snr = hs.to(dev, non_blocking=True)
            gains = torch.empty(plan.S, device=dev)
            y = torch.empty(plan.y_size, device=dev)
            tl = torch.empty(plan.R, dtype=torch.int32, device=dev)
            plan.filter_mix(x, rir, gains, y, snr_db=snr, trunc_len=tl)
            res = {"y": y, "gains": gains, "trunc_len": tl}
            if gy is not None:
                g = hg.to(dev, non_blocking=True)
                gx, gr, gg = torch.empty_like(x), torch.empty_like(rir), torch.empty_like(gains)
                plan.filter_mix_backward(g, x, gains, gx, gr, gg)
                res.update(grad_x=gx, grad_rir=gr, grad_gains=gg)
            host = {k: v.to("cpu", non_blocking=True) for k, v in res.items()} if self.keep else \
                {"trunc_len": tl.to("cpu", non_blocking=True)}
            e1.record(stream)
            plan.sync_status()
            e1.synchronize()
            wall = (time.perf_counter() - t0) * 1e3
            q = plan.query()
            sizes, cnt = np.unique(1 << q["log2_n"].astype(np.int64), return_counts=True)
            bufs = 4 * (x.numel() + rir.numel() + y.numel() + 2 * gains.numel())
            if gy is not None:
                bufs += 4 * (g.numel() + gx.numel() + gr.numel())
            records.append(BatchRecord(grp, float(np.sum(sub.num_samples)) / synth.FS, wall,
                                       e0.elapsed_time(e1), plan_ms, int(bufs + plan.scratch_bytes),
                                       {int(k): int(c) for k, c in zip(sizes, cnt)}, q,
                                       host["trunc_len"].numpy().copy()))
            if self.keep:
                outputs.append({k: v.numpy() for k, v in host.items()})
            plan.close()
        return StreamResult(records, outputs)
