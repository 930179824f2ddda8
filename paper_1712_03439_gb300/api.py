"""Python front end of the rsim C-ABI.

Argument marshalling only: torch tensors provide device memory and the
current CUDA stream; every step of the computation runs in librsim.so.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _lib


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _want(t, n, dtype, name):
    if t is None:
        return
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name}: expected a contiguous {dtype} tensor of {n} elements, "
                         f"got {t.dtype} {tuple(t.shape)}")


class Plan:
    """A plan for a batch shape: utterance lengths, sources per utterance,
    microphones and RIR lengths (see rsim_plan in include/rsim.h)."""

    def __init__(self, num_sources, num_samples, rir_len, num_mics, eta_db=20.0,
                 fft_sizes=None, gain_mode=0, segment_len=0, bwd_segment_len=0, fft_cost=None,
                 device=None, graphs=True, output_mode=0, snr_ref_mic=0, rooms=False, long_rirs=False,
                 spectrum_cache=True):
        self._lib = _lib.load()
        self._handle = None
        self.num_sources = np.ascontiguousarray(num_sources, dtype=np.int32)
        self.num_samples = np.ascontiguousarray(num_samples, dtype=np.int64)
        self.rir_len = np.ascontiguousarray(rir_len, dtype=np.int32)
        self.num_mics = int(num_mics)
        self.gain_mode = int(gain_mode)
        self.output_mode = int(output_mode)
        self.eta_db = float(eta_db)
        self.spectrum_cache = bool(spectrum_cache)
        mask = 0
        for n in (fft_sizes or []):
            m = int(round(math.log2(n)))
            if 1 << m != n:
                raise ValueError(f"FFT size {n} is not a power of two")
            mask |= 1 << m
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        # measured per-size costs and tile lengths for this GPU, if tuned
        from .autotune import load_table
        tuned = load_table(torch.cuda.get_device_name(self.device)) or {}
        if fft_cost is None and "fft_cost_ns" in tuned:
            fft_cost = {int(k): float(v) for k, v in tuned["fft_cost_ns"].items()}
        if not segment_len:
            segment_len = int(tuned.get("segment_len", 0))
        self.tuned = bool(tuned)
        self._cost = None
        if fft_cost is not None:
            self._cost = np.zeros(32, np.float32)
            for n, c in dict(fft_cost).items():
                self._cost[int(round(math.log2(n)))] = c
        self._fixed = dict(num_mics=self.num_mics, eta_db=self.eta_db, fft_sizes_mask=mask,
                           gain_mode=self.gain_mode, segment_len=int(segment_len),
                           bwd_segment_len=int(bwd_segment_len), disable_graphs=0 if graphs else 1,
                           output_mode=self.output_mode, snr_ref_mic=int(snr_ref_mic), rooms=1 if rooms else 0,
                           long_rirs=1 if long_rirs else 0, spectrum_cache=1 if spectrum_cache else 0)
        h = ctypes.c_void_p()
        _lib.check(self._lib, self._lib.rsim_plan(ctypes.byref(self._desc()), self.device, ctypes.byref(h)))
        self._handle = h
        self._set_shape()
        # FFT sizes the plan may pick (one forward/backward launch each)
        self.num_fft_sizes = bin(mask).count("1") if mask else 4

    def _desc(self):
        return _lib.PlanDesc(num_utts=self.num_sources.shape[0], num_sources=self.num_sources.ctypes.data,
                             num_samples=self.num_samples.ctypes.data, rir_len=self.rir_len.ctypes.data,
                             fft_cost=None if self._cost is None else self._cost.ctypes.data, **self._fixed)

    def _set_shape(self):
        self.U = int(self.num_sources.shape[0])
        self.S = int(self.num_sources.sum())
        self.R = int(self.rir_len.shape[0])
        self.x_size = int(np.sum(self.num_sources.astype(np.int64) * self.num_samples))
        # output samples per mic: Nx, or Nx + (longest RIR of the utterance) - 1
        self.num_out = self.num_samples.copy()
        if self.output_mode:
            r0 = np.concatenate([[0], np.cumsum(self.num_sources.astype(np.int64) * self.num_mics)])
            self.num_out += np.array([self.rir_len[r0[u]:r0[u + 1]].max() for u in range(self.U)],
                                     dtype=np.int64) - 1
        self.y_size = int(np.sum(self.num_out) * self.num_mics)
        self.rir_size = int(np.sum(self.rir_len.astype(np.int64)))
        # gains: one per source, or one per (source, microphone) in gain mode 2
        self.G = self.R if self.gain_mode == 2 else self.S
        # forwards run on this plan so far: the backward uses the state (cut-off
        # lengths, RIR spectra, the RIR buffer) of the most recent one
        self.forward_count = 0

    def reshape(self, num_sources, num_samples, rir_len):
        """rsim_plan_reshape: this plan, re-planned in place for another batch shape
        that fits its shape class (raises RsimError with status 2 when it does not;
        the plan then keeps its shape)."""
        old = (self.num_sources, self.num_samples, self.rir_len)
        self.num_sources = np.ascontiguousarray(num_sources, dtype=np.int32)
        self.num_samples = np.ascontiguousarray(num_samples, dtype=np.int64)
        self.rir_len = np.ascontiguousarray(rir_len, dtype=np.int32)
        try:
            _lib.check(self._lib, self._lib.rsim_plan_reshape(self._handle, ctypes.byref(self._desc())))
        except Exception:
            self.num_sources, self.num_samples, self.rir_len = old
            raise
        self._set_shape()

    def reshape_for(self, batch):
        self.reshape(batch.num_sources, batch.num_samples, batch.rir_len)

    @classmethod
    def for_batch(cls, batch, **kw):
        return cls(batch.num_sources, batch.num_samples, batch.rir_len, batch.num_mics, **kw)

    # ------------------------------------------------------------------
    def filter_mix(self, x, rir, gains, y, snr_db=None, trunc_len=None, energy_kept_frac=None,
                   stream=None):
        """rsim_filter_mix: writes y (and gains when gain_mode = 0)."""
        _want(x, self.x_size, torch.float32, "x")
        _want(rir, self.rir_size, torch.float32, "rir")
        _want(gains, self.G, torch.float32, "gains")
        _want(y, self.y_size, torch.float32, "y")
        _want(snr_db, self.S, torch.float32, "snr_db")
        _want(trunc_len, self.R, torch.int32, "trunc_len")
        _want(energy_kept_frac, self.R, torch.float32, "energy_kept_frac")
        st = self._lib.rsim_filter_mix(self._handle, _stream(stream), _ptr(x), _ptr(rir),
                                       _ptr(snr_db), _ptr(gains), _ptr(y), _ptr(trunc_len),
                                       _ptr(energy_kept_frac))
        _lib.check(self._lib, st)
        self.forward_count += 1

    def filter_mix_rooms(self, x, geom, gains, y, snr_db=None, trunc_len=None, energy_kept_frac=None,
                         rir_out=None, order=8, fs=16000.0, c0=343.0, stream=None):
        """rsim_filter_mix_rooms: the forward with the RIRs made on the device from
        room geometry (geom: float32 CUDA tensor [R, 10], rows of room (3),
        source (3), microphone (3), r); needs a plan made with rooms=True."""
        _want(x, self.x_size, torch.float32, "x")
        if not isinstance(geom, torch.Tensor) or not geom.is_cuda or geom.dtype != torch.float32 \
                or not geom.is_contiguous() or tuple(geom.shape) != (self.R, 10):
            raise ValueError(f"geom must be a contiguous float32 CUDA tensor of shape [{self.R}, 10]")
        _want(gains, self.G, torch.float32, "gains")
        _want(y, self.y_size, torch.float32, "y")
        _want(snr_db, self.S, torch.float32, "snr_db")
        _want(trunc_len, self.R, torch.int32, "trunc_len")
        _want(energy_kept_frac, self.R, torch.float32, "energy_kept_frac")
        _want(rir_out, self.rir_size, torch.float32, "rir_out")
        st = self._lib.rsim_filter_mix_rooms(self._handle, _stream(stream), _ptr(x), _ptr(geom), int(order),
                                             float(fs), float(c0), _ptr(snr_db), _ptr(gains), _ptr(y),
                                             _ptr(trunc_len), _ptr(energy_kept_frac), _ptr(rir_out))
        _lib.check(self._lib, st)
        self.forward_count += 1

    def filter_mix_backward(self, grad_y, x, gains, grad_x, grad_rir, grad_gains, stream=None):
        """rsim_filter_mix_backward: writes grad_x (if given), grad_rir and grad_gains."""
        _want(grad_y, self.y_size, torch.float32, "grad_y")
        _want(x, self.x_size, torch.float32, "x")
        _want(gains, self.G, torch.float32, "gains")
        _want(grad_x, self.x_size, torch.float32, "grad_x")
        _want(grad_rir, self.rir_size, torch.float32, "grad_rir")
        _want(grad_gains, self.G, torch.float32, "grad_gains")
        st = self._lib.rsim_filter_mix_backward(self._handle, _stream(stream), _ptr(grad_y), _ptr(x),
                                                _ptr(gains), _ptr(grad_x), _ptr(grad_rir),
                                                _ptr(grad_gains))
        _lib.check(self._lib, st)

    def sync_status(self, stream=None):
        _lib.check(self._lib, self._lib.rsim_plan_sync_status(self._handle, _stream(stream)))

    def query(self, stream=None):
        """Per-utterance plan of the last forward: log2 N, hop, L_max, blocks."""
        out = {k: np.zeros(self.U, np.int32) for k in ("log2_n", "hop", "l_max", "num_blocks")}
        st = self._lib.rsim_plan_query(self._handle, _stream(stream),
                                       *(ctypes.c_void_p(out[k].ctypes.data)
                                         for k in ("log2_n", "hop", "l_max", "num_blocks")))
        _lib.check(self._lib, st)
        return out

    def set_timing(self, enable: bool):
        _lib.check(self._lib, self._lib.rsim_plan_set_timing(self._handle, int(bool(enable))))

    def stage_times(self):
        """{stage: (total ms, calls)} recorded since the last query (synchronises)."""
        ms = np.zeros(len(_lib.STAGES), np.float64)
        calls = np.zeros(len(_lib.STAGES), np.int32)
        _lib.check(self._lib, self._lib.rsim_plan_stage_times(
            self._handle, ctypes.c_void_p(ms.ctypes.data), ctypes.c_void_p(calls.ctypes.data)))
        return {k: (float(ms[i]), int(calls[i])) for i, k in enumerate(_lib.STAGES)}

    # ------------------------------------------------------------------
    @staticmethod
    def mel_desc(channel=0, hop=160, fs=16000.0, n_mels=128, f_lo=125.0, f_hi=7500.0, log_floor=1e-6,
                 stack=4, stride=3):
        """The log-Mel description (defaults: the paper's features at 16 kHz)."""
        return _lib.MelDesc(channel=int(channel), hop=int(hop), fs=float(fs), n_mels=int(n_mels),
                            f_lo=float(f_lo), f_hi=float(f_hi), log_floor=float(log_floor), stack=int(stack),
                            stride=int(stride))

    def log_mel_rows(self, **kw):
        """(rows per utterance [U], total rows) of log_mel's output."""
        d = self.mel_desc(**kw)
        rows = np.zeros(self.U, np.int64)
        total = ctypes.c_int64()
        _lib.check(self._lib, self._lib.rsim_plan_log_mel_rows(self._handle, ctypes.byref(d),
                                                               ctypes.c_void_p(rows.ctypes.data),
                                                               ctypes.byref(total)))
        return rows, int(total.value)

    def log_mel(self, y, feats=None, stream=None, **kw):
        """rsim_plan_log_mel: stacked log-Mel features of one microphone of y.
        Returns feats [rows, stack * n_mels] (allocated if not given)."""
        d = self.mel_desc(**kw)
        _want(y, self.y_size, torch.float32, "y")
        _, total = self.log_mel_rows(**kw)
        width = d.stack * d.n_mels
        if feats is None:
            feats = torch.empty((total, width), dtype=torch.float32, device=y.device)
        _want(feats.view(-1), total * width, torch.float32, "feats")
        _lib.check(self._lib, self._lib.rsim_plan_log_mel(self._handle, _stream(stream), _ptr(y), ctypes.byref(d),
                                                          _ptr(feats)))
        return feats

    @property
    def scratch_bytes(self) -> int:
        return int(self._lib.rsim_plan_scratch_bytes(self._handle))

    def close(self):
        if self._handle is not None:
            self._lib.rsim_plan_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def source_gains_noalloc(num_sources, num_samples, x, snr_db, gains, stream=None):
    """rsim_source_gains_noalloc: the gain_mode = 0 gains without a plan and
    without any device allocation (scratch is a fixed array in the library)."""
    lib = _lib.load()
    ns = np.ascontiguousarray(num_sources, dtype=np.int32)
    nx = np.ascontiguousarray(num_samples, dtype=np.int64)
    S = int(ns.sum())
    _want(x, int(np.sum(ns.astype(np.int64) * nx)), torch.float32, "x")
    _want(snr_db, S, torch.float32, "snr_db")
    _want(gains, S, torch.float32, "gains")
    st = lib.rsim_source_gains_noalloc(_stream(stream), ns.shape[0], ctypes.c_void_p(ns.ctypes.data),
                                       ctypes.c_void_p(nx.ctypes.data), _ptr(x), _ptr(snr_db), _ptr(gains))
    _lib.check(lib, st)


# image-method RIRs: bits of the status word rsim_image_rirs writes
IMAGE_BAD_GEOMETRY = 1
IMAGE_BAD_LENGTH = 2


def image_rirs(geom, rir_off, max_len, rir, order=8, fs=16000.0, c0=343.0, status=None, stream=None):
    """rsim_image_rirs: Eq. 1 RIRs for R (source, microphone) pairs.

    geom      float32 CUDA tensor [R, 10]: room (3), source (3), microphone (3), r
    rir_off   int64 CUDA tensor [R + 1]: RIR r is rir[rir_off[r]:rir_off[r + 1]]
    max_len   the longest RIR (host int; sizes the launch)
    rir       float32 CUDA tensor, written
    status    optional int32 CUDA tensor [1]: IMAGE_BAD_GEOMETRY / IMAGE_BAD_LENGTH bits"""
    lib = _lib.load()
    if not isinstance(geom, torch.Tensor) or not geom.is_cuda or geom.dtype != torch.float32 \
            or not geom.is_contiguous() or geom.dim() != 2 or geom.shape[1] != 10:
        raise ValueError("geom must be a contiguous float32 CUDA tensor of shape [R, 10]")
    R = int(geom.shape[0])
    _want(rir_off, R + 1, torch.int64, "rir_off")
    if not isinstance(rir, torch.Tensor) or not rir.is_cuda or rir.dtype != torch.float32 \
            or not rir.is_contiguous():
        raise ValueError("rir must be a contiguous float32 CUDA tensor")
    _want(status, 1, torch.int32, "status")
    st = lib.rsim_image_rirs(_stream(stream), R, _ptr(geom), _ptr(rir_off), int(max_len), int(order),
                             float(fs), float(c0), _ptr(rir), _ptr(status))
    _lib.check(lib, st)


# ---------------------------------------------------------------------------
# convenience and autograd
# ---------------------------------------------------------------------------
def filter_mix(plan: Plan, x, rir, snr_db=None, gains=None, stream=None):
    """Allocates outputs and runs the forward.  Returns dict(y, gains, trunc_len,
    energy_kept_frac)."""
    dev = x.device
    y = torch.empty(plan.y_size, dtype=torch.float32, device=dev)
    if gains is None:
        gains = torch.empty(plan.G, dtype=torch.float32, device=dev)
    tl = torch.empty(plan.R, dtype=torch.int32, device=dev)
    ekf = torch.empty(plan.R, dtype=torch.float32, device=dev)
    plan.filter_mix(x, rir, gains, y, snr_db=snr_db, trunc_len=tl, energy_kept_frac=ekf,
                    stream=stream)
    return dict(y=y, gains=gains, trunc_len=tl, energy_kept_frac=ekf)


class RsimFilterMix(torch.autograd.Function):
    """y = filter_mix(x, rir, gains) with the hand-written adjoint.

    The plan must use gain_mode 1 (gains [S], one per source) or 2 (gains [R],
    one per source and microphone): gains are an input.  The truncation is a
    fixed mask: grad_rir is zero beyond each kept length.

    The library's backward reuses the state of the plan's most recent forward
    (cut-off lengths, cached RIR spectra and, with per-(i, j) gains, the RIR
    buffer that forward read).  The tensors this forward used (x, the
    contiguous rir, gains) are saved, so that buffer stays alive; when another
    forward ran on the same plan in between (gradient accumulation, a second
    branch), the backward first re-runs this call's forward on the saved
    tensors to restore that state."""

    @staticmethod
    def forward(ctx, plan, x, rir, gains):
        if plan.gain_mode not in (1, 2):
            raise ValueError("RsimFilterMix needs a plan with gain_mode 1 or 2")
        x, rir, gains = x.contiguous(), rir.contiguous(), gains.contiguous()
        y = torch.empty(plan.y_size, dtype=torch.float32, device=x.device)
        plan.filter_mix(x, rir, gains, y)
        ctx.plan = plan
        ctx.forward_count = plan.forward_count
        ctx.save_for_backward(x, rir, gains)
        return y

    @staticmethod
    def backward(ctx, grad_y):
        plan = ctx.plan
        x, rir, gains = ctx.saved_tensors
        if plan.forward_count != ctx.forward_count:
            # a later forward replaced the plan's state: rebuild this call's
            plan.filter_mix(x, rir, gains, torch.empty(plan.y_size, dtype=torch.float32, device=x.device))
            ctx.forward_count = plan.forward_count
        grad_y = grad_y.contiguous()
        gx = torch.empty(plan.x_size, dtype=torch.float32, device=x.device) if ctx.needs_input_grad[1] else None
        gr = torch.empty(plan.rir_size, dtype=torch.float32, device=x.device)
        gg = torch.empty(plan.G, dtype=torch.float32, device=x.device)
        plan.filter_mix_backward(grad_y, x, gains, gx, gr, gg)
        return None, gx, gr, gg


def filter_mix_autograd(plan: Plan, x, rir, gains):
    return RsimFilterMix.apply(plan, x, rir, gains)
