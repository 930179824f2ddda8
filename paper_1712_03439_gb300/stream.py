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
    scratch += 8 * rir_sum + 8                           # RIR-gradient partials (twice the taps), prefix
    scratch += 8 * n_src * (-(-nx // _POWER_CHUNK))      # power partial sums
    scratch += 4 * 3 * 4 * max(nseg, n_src * n_mics) + 256
    # backward streams: order and cost prefix per size, first and last piece, one piece
    # with its partial offset and source-gain partials
    scratch += n_src * (4 * 4 + 8 * 4 + 4 + 4 + 8 + 4 * 16)
    return int(buf + scratch)


def partition_bytes(utt_taps_max: int = 0, ctas: int = PART_CTAS) -> int:
    """The backward partition's per-CTA scratch: one extra piece per CTA boundary
    (partial offset and source-gain partials; its RIR-gradient partials are in
    the utterances' share) and the chunk starts."""
    return int(ctas * (8 + 4 * 16 + 3 * 4) + 4096)


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
    wall_ms: float          # inputs in pinned host memory to results on the host
    device_ms: float        # first host-to-device copy to last device-to-host copy
    plan_ms: float          # re-planning the shape-class plan for the batch (or making a plan)
    footprint_bytes: int    # buffers + the plan's real scratch
    fft_blocks: dict        # FFT size -> utterances that used it
    query: dict             # the plan's per-utterance choice (log2 N, hop, L_max, blocks)
    trunc_len: np.ndarray   # kept RIR lengths of the batch
    staging_ms: float = 0.0  # host copy of the inputs into pinned memory (overlapped with the
                             # previous batch's device work)
    reshaped: bool = True    # served by the shape-class plan (False: a plan made for it)


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
                 output_mode: int = 0, device=None, keep_outputs: bool = True, class_plan: bool = True,
                 **plan_kw):
        import torch
        self.torch = torch
        self.budget = int(budget_bytes)
        self.eta_db = float(eta_db)
        self.backward = bool(backward)
        self.output_mode = int(output_mode)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.keep = keep_outputs
        self.class_plan = bool(class_plan)   # one shape-class plan, re-planned per batch
        # one call per plan: launch eagerly rather than capture a graph that is never replayed;
        # no spectrum cache: its memory (up to 16 bytes per source sample) would shrink the
        # batches the budget admits, and a batch here is small next to the copies around it
        self.plan_kw = dict(dict(graphs=False, spectrum_cache=False), **plan_kw)
        self._pin = {}

    def _staging(self, name, n, dtype):
        t = self._pin.get(name)
        if t is None or t.numel() < n or t.dtype != dtype:
            t = self.torch.empty(max(n, 1), dtype=dtype, pin_memory=True)
            self._pin[name] = t
        return t[:n]

    @staticmethod
    def shape_class(batch: synth.Batch, groups):
        """Arrays (num_sources, num_samples, rir_len) of an upper-bound batch for the
        groups: the group with the most samples, padded (one single-source
        utterance with the missing samples and RIR taps, then tiny utterances) so
        that its utterance, source and RIR counts, samples, RIR taps, segments and
        power-scan chunks (sources x chunks of the longest utterance) reach every
        group's."""
        J = batch.num_mics
        ri = batch.rir_index()
        if len(groups) == 1:
            g0 = list(groups[0])
            return (batch.num_sources[g0].astype(np.int32), batch.num_samples[g0].astype(np.int64),
                    np.concatenate([batch.rir_len[ri[u]:ri[u + 1]] for u in g0]).astype(np.int32))

        def stats(g):
            g = list(g)
            ns = batch.num_sources[g].astype(np.int64)
            nx = batch.num_samples[g].astype(np.int64)
            taps = int(sum(int(batch.rir_len[ri[u]:ri[u + 1]].sum()) for u in g))
            return dict(U=len(g), S=int(ns.sum()), X=int(np.sum(ns * nx)), Y=int(nx.sum()), T=taps,
                        G=int(np.sum(-(-nx // 16384))), C=int(ns.sum()) * int(-(-nx.max() // _POWER_CHUNK)))
        st = [stats(g) for g in groups]
        big = max(range(len(groups)), key=lambda k: st[k]["X"])
        need = {k: max(x[k] for x in st) for k in st[0]}
        g0 = list(groups[big])
        ns = [int(batch.num_sources[u]) for u in g0]
        nx = [int(batch.num_samples[u]) for u in g0]
        rl = [int(v) for u in g0 for v in batch.rir_len[ri[u]:ri[u + 1]]]
        # the missing samples and taps on one single-source utterance
        extra_x = max(0, need["X"] - st[big]["X"], need["Y"] - st[big]["Y"])
        extra_t = max(0, need["T"] - st[big]["T"])
        ns.append(1)
        nx.append(max(1, extra_x))
        rl += [max(1, extra_t)] + [1] * (J - 1)
        # tiny utterances for the counts, the segments and the power-scan chunks
        ch = -(-max(nx) // _POWER_CHUNK)
        seg = sum(-(-v // 16384) for v in nx)
        n_tiny = max(0, need["U"] - len(ns), need["S"] - sum(ns), need["G"] - seg, -(-need["C"] // ch) - sum(ns))
        ns += [1] * n_tiny
        nx += [1] * n_tiny
        rl += [1] * (n_tiny * J)
        return np.array(ns, np.int32), np.array(nx, np.int64), np.array(rl, np.int32)

    def run(self, batch: synth.Batch, grad_y=None, groups=None) -> StreamResult:
        """grad_y(sub_batch, ny) -> float32 upstream gradient for a batch (or None:
        a seeded one).  Returns per-batch records and (if kept) outputs.

        One plan serves the run: made once for an upper-bound shape of all the
        admitted batches (shape_class) and re-planned in place for each batch
        (Plan.reshape: no allocation); a batch that does not fit gets a plan of its
        own.  A host thread copies the next batch's inputs into the other of two
        pinned staging sets while the current batch runs on the device."""
        import threading
        torch = self.torch
        from ._lib import RsimError
        from .api import Plan
        dev = self.device
        stream = torch.cuda.current_stream(dev)
        def class_bytes(cns, cnx, crl):
            r0 = np.concatenate([[0], np.cumsum(cns.astype(np.int64) * batch.num_mics)])
            taps = [int(crl[r0[u]:r0[u + 1]].sum()) for u in range(len(cns))]
            return PLAN_FIXED_BYTES + partition_bytes() + sum(
                utterance_bytes(int(cnx[u]), int(cns[u]), batch.num_mics, taps[u],
                                int(crl[r0[u]:r0[u + 1]].max()), backward=self.backward,
                                output_mode=self.output_mode) for u in range(len(cns)))
        # the class plan's estimated footprint (its buffers bound every batch's) must fit
        # the budget: batches are admitted with the largest share of the budget that
        # leaves room for the class's padding; without one, every batch gets its own plan
        cls = None
        if groups is None and not self.class_plan:
            groups = admit(batch, self.budget, backward=self.backward, output_mode=self.output_mode)
        elif groups is None:
            for frac in (0.9, 0.8, 0.7, 0.6):
                g = admit(batch, int(frac * self.budget), backward=self.backward, output_mode=self.output_mode)
                c = self.shape_class(batch, g) if g else None
                if c is not None and (len(g) == 1 or class_bytes(*c) <= self.budget):
                    groups, cls = g, c
                    break
            if groups is None:
                groups = admit(batch, self.budget, backward=self.backward, output_mode=self.output_mode)
        elif self.class_plan:
            c = self.shape_class(batch, list(groups)) if len(groups) else None
            if c is not None and (len(groups) == 1 or class_bytes(*c) <= self.budget):
                cls = c
        groups = list(groups)
        cls_plan = None
        if cls is not None:
            cls_plan = Plan(*cls, batch.num_mics, eta_db=self.eta_db, output_mode=self.output_mode,
                            device=dev.index, **self.plan_kw)
        subs = [batch.subset(g) for g in groups]

        def inputs(gi):
            sub = subs[gi]
            ny = synth.output_lengths(sub, self.output_mode)
            gy = (grad_y(sub, ny) if grad_y is not None
                  else synth.grad_like(1000 + gi, int(ny.sum()) * sub.num_mics)) if self.backward else None
            return sub, gy

        # two pinned staging sets; set k % 2 holds batch k until its copies to the device are done
        copied = [None, None]                   # events after each set's host-to-device copies

        def stage(gi, sub, gy, out):
            k = gi % 2
            t = time.perf_counter()
            if copied[k] is not None:
                copied[k].synchronize()
            hx = self._staging(f"x{k}", sub.x.size, torch.float32)
            hr = self._staging(f"rir{k}", sub.rir.size, torch.float32)
            hs = self._staging(f"snr{k}", sub.snr_db.size, torch.float32)
            hx.numpy()[:sub.x.size] = sub.x
            hr.numpy()[:sub.rir.size] = sub.rir
            hs.numpy()[:sub.snr_db.size] = sub.snr_db
            hg = None
            if gy is not None:
                hg = self._staging(f"gy{k}", gy.size, torch.float32)
                hg.numpy()[:gy.size] = gy
            out.update(hx=hx, hr=hr, hs=hs, hg=hg, ms=(time.perf_counter() - t) * 1e3)

        records, outputs = [], []
        nxt = {}
        if groups:
            s0, g0 = inputs(0)
            stage(0, s0, g0, nxt)
        for gi, grp in enumerate(groups):
            cur, nxt = nxt, {}
            sub = subs[gi]
            gy_sz = int(synth.output_lengths(sub, self.output_mode).sum()) * sub.num_mics if self.backward else 0
            worker = None
            if gi + 1 < len(groups):
                s1, g1 = inputs(gi + 1)
                worker = threading.Thread(target=stage, args=(gi + 1, s1, g1, nxt))
            # the batch's latency runs from here: its inputs are in pinned host memory
            t0 = time.perf_counter()
            tp = time.perf_counter()
            plan, reshaped = cls_plan, cls_plan is not None
            if reshaped:
                try:
                    plan.reshape_for(sub)
                except RsimError as e:
                    if e.status != 2:
                        raise
                    reshaped = False
            if not reshaped:
                plan = Plan.for_batch(sub, eta_db=self.eta_db, output_mode=self.output_mode, device=dev.index,
                                      **self.plan_kw)
            plan_ms = (time.perf_counter() - tp) * 1e3
            e0, e1, ec = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
                          torch.cuda.Event())
            e0.record(stream)
            x = cur["hx"][:sub.x.size].to(dev, non_blocking=True)
            rir = cur["hr"][:sub.rir.size].to(dev, non_blocking=True)
            snr = cur["hs"][:sub.snr_db.size].to(dev, non_blocking=True)
            g = cur["hg"][:gy_sz].to(dev, non_blocking=True) if cur["hg"] is not None else None
            ec.record(stream)
            copied[gi % 2] = ec
            gains = torch.empty(plan.S, device=dev)
            y = torch.empty(plan.y_size, device=dev)
            tl = torch.empty(plan.R, dtype=torch.int32, device=dev)
            plan.filter_mix(x, rir, gains, y, snr_db=snr, trunc_len=tl)
            res = {"y": y, "gains": gains, "trunc_len": tl}
            if g is not None:
                gx, gr, gg = torch.empty_like(x), torch.empty_like(rir), torch.empty_like(gains)
                plan.filter_mix_backward(g, x, gains, gx, gr, gg)
                res.update(grad_x=gx, grad_rir=gr, grad_gains=gg)
            host = {k: v.to("cpu", non_blocking=True) for k, v in res.items()} if self.keep else \
                {"trunc_len": tl.to("cpu", non_blocking=True)}
            e1.record(stream)
            if worker is not None:
                worker.start()                 # the next batch is staged while this one runs
            plan.sync_status()
            e1.synchronize()
            wall = (time.perf_counter() - t0) * 1e3
            q = plan.query()
            sizes, cnt = np.unique(1 << q["log2_n"].astype(np.int64), return_counts=True)
            bufs = 4 * (x.numel() + rir.numel() + y.numel() + 2 * gains.numel())
            if g is not None:
                bufs += 4 * (g.numel() + gx.numel() + gr.numel())
            records.append(BatchRecord(grp, float(np.sum(sub.num_samples)) / synth.FS, wall,
                                       e0.elapsed_time(e1), plan_ms, int(bufs + plan.scratch_bytes),
                                       {int(k): int(c) for k, c in zip(sizes, cnt)}, q,
                                       host["trunc_len"].numpy().copy(), cur["ms"], reshaped))
            if self.keep:
                outputs.append({k: v.numpy() for k, v in host.items()})
            if worker is not None:
                worker.join()
            if not reshaped:
                plan.close()
        if cls_plan is not None:
            cls_plan.close()
        return StreamResult(records, outputs)
