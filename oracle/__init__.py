"""ctypes front end of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this package; the library under
``paper_1712_03439_gb300`` never does.  It shares no code with the CUDA path.

Batch arguments are duck-typed: any object with ``num_mics``,
``num_sources`` (int32 [U]), ``num_samples`` (int64 [U]), ``rir_len``
(int32 [R]), ``x``, ``rir`` and ``snr_db`` (float32, packed as described in
the library header) works.  All arithmetic is FP64; FP32 inputs are converted
exactly.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

_CFLAGS = ["-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
           "-D_DEFAULT_SOURCE"]


def build_library(force: bool = False, extra_flags=()) -> str:
    """Compiles oracle.c into liboracle.so (gcc, OpenMP).  Returns the path."""
    out = _LIB_PATH
    if extra_flags:
        tag = "_".join(f.strip("-").replace("=", "") for f in extra_flags)
        out = os.path.join(_HERE, f"liboracle_{tag}.so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        cmd = ["gcc", *_CFLAGS, *extra_flags, _SRC, "-o", out, "-lm"]
        subprocess.run(cmd, check=True)
    return out


def _load(path=None):
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        override = os.environ.get("ORACLE_LIB")
        _lib = _bind(ctypes.CDLL(override if override else build_library()))
    return _lib


def _bind(lib):
    P = ctypes.c_void_p
    i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.oracle_cost_td.restype = f64
    lib.oracle_cost_td.argtypes = [f64, f64, f64, f64]
    lib.oracle_cost_fft.restype = f64
    lib.oracle_cost_fft.argtypes = [f64, f64, f64]
    lib.oracle_cost_ola.restype = f64
    lib.oracle_cost_ola.argtypes = [f64, f64, f64, f64, f64]
    lib.oracle_best_ola_n.restype = i64
    lib.oracle_best_ola_n.argtypes = [f64, f64, f64, f64, ctypes.c_int, ctypes.c_int]
    lib.oracle_truncate.restype = i64
    lib.oracle_truncate.argtypes = [P, i64, f64, P, P, P]
    lib.oracle_gains.restype = ctypes.c_int
    lib.oracle_gains.argtypes = [P, i64, i32, P, P]
    lib.oracle_mix_direct.restype = None
    lib.oracle_mix_direct.argtypes = [P, i64, i32, i32, P, P, P, P, P]
    lib.oracle_truncate_batch.restype = ctypes.c_int
    lib.oracle_truncate_batch.argtypes = [i64, P, P, f64, P, P, P, P, ctypes.c_int]
    lib.oracle_forward_batch.restype = ctypes.c_int
    lib.oracle_forward_batch.argtypes = [i32, i32, P, P, P, P, P, P, P, ctypes.c_int, P, P,
                                         ctypes.c_int, ctypes.c_int]
    lib.oracle_backward_batch.restype = ctypes.c_int
    lib.oracle_backward_batch.argtypes = [i32, i32, P, P, P, P, P, P, P, P, P, P, P,
                                          ctypes.c_int, ctypes.c_int]
    lib.oracle_mix_ola.restype = ctypes.c_int
    lib.oracle_mix_ola.argtypes = [P, i64, i32, i32, P, P, P, P, i64, P]
    lib.oracle_forward_ola_batch.restype = ctypes.c_int
    lib.oracle_forward_ola_batch.argtypes = [i32, i32, P, P, P, P, P, P, P, i64, P,
                                             ctypes.c_int]
    lib.oracle_mix_window.restype = None
    lib.oracle_mix_window.argtypes = [P, i64, i32, i32, P, P, P, P, i64, i64, P]
    lib.oracle_dh_window.restype = None
    lib.oracle_dh_window.argtypes = [P, i64, P, i64, i64, ctypes.c_double, i64, i64, P]
    lib.oracle_dx_window.restype = None
    lib.oracle_dx_window.argtypes = [P, i64, i32, i32, P, P, P, ctypes.c_double, i64, i64, P]
    lib.oracle_dft_real.restype = None
    lib.oracle_dft_real.argtypes = [P, i64, i64, P, P]
    lib.oracle_max_threads.restype = ctypes.c_int
    lib.oracle_max_threads.argtypes = []
    lib.oracle_image_list.restype = i64
    lib.oracle_image_list.argtypes = [P, P, P, ctypes.c_float, i32, ctypes.c_float, ctypes.c_float,
                                      P, P, P, P, P]
    lib.oracle_image_rir.restype = i64
    lib.oracle_image_rir.argtypes = [P, P, P, ctypes.c_float, i32, ctypes.c_float, ctypes.c_float,
                                     i64, P]
    lib.oracle_hz_to_mel.restype = f64
    lib.oracle_hz_to_mel.argtypes = [f64]
    lib.oracle_mel_to_hz.restype = f64
    lib.oracle_mel_to_hz.argtypes = [f64]
    lib.oracle_mel_filters.restype = None
    lib.oracle_mel_filters.argtypes = [i32, f64, i32, f64, f64, P]
    lib.oracle_frame_power.restype = None
    lib.oracle_frame_power.argtypes = [P, i32, P]
    lib.oracle_log_mel_rows.restype = i64
    lib.oracle_log_mel_rows.argtypes = [i64, i32, i32, i32, i32]
    lib.oracle_log_mel.restype = i64
    lib.oracle_log_mel.argtypes = [P, i64, i32, i32, f64, i32, f64, f64, f64, i32, i32, P]
    lib.oracle_log_mel_batch.restype = None
    lib.oracle_log_mel_batch.argtypes = [i32, i32, P, P, i32, i32, i32, f64, i32, f64, f64, f64, i32, i32, P, P,
                                         ctypes.c_int]
    lib.oracle_image_rirs.restype = None
    lib.oracle_image_rirs.argtypes = [i64, P, P, i32, ctypes.c_float, ctypes.c_float, P, P,
                                      ctypes.c_int]
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


class OracleError(RuntimeError):
    pass


# ---- cost models (Eq. 3, 5, 6) -------------------------------------------------
def cost_td(I, J, Nx, Nh, lib=None):
    return (lib or _load()).oracle_cost_td(I, J, Nx, Nh)


def cost_fft(I, J, N, lib=None):
    return (lib or _load()).oracle_cost_fft(I, J, N)


def cost_ola(I, J, Nx, Nh, N, lib=None):
    return (lib or _load()).oracle_cost_ola(I, J, Nx, Nh, N)


def best_ola_n(I, J, Nx, Nh, m_lo=6, m_hi=20, lib=None):
    return int((lib or _load()).oracle_best_ola_n(I, J, Nx, Nh, m_lo, m_hi))


def max_threads(lib=None) -> int:
    return int((lib or _load()).oracle_max_threads())


# ---- single-RIR / single-utterance entry points ----------------------------
def truncate(h, eta_db, lib=None):
    """Eq. 7-9 on one RIR.  Returns (L, peak, e_tot, e_kept)."""
    h = _f64(h)
    pk, et, ek = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    L = (lib or _load()).oracle_truncate(_p(h), h.shape[0], float(eta_db), ctypes.byref(pk),
                                         ctypes.byref(et), ctypes.byref(ek))
    if L < 0:
        raise OracleError("invalid truncation arguments")
    return int(L), pk.value, et.value, ek.value


def gains(x_sources, snr_db, lib=None):
    """Per-source gains for one utterance.  x_sources: [I, Nx]."""
    x = _f64(x_sources)
    I, nx = x.shape
    snr = _f64(snr_db)
    alpha = np.zeros(I)
    rc = (lib or _load()).oracle_gains(_p(x), nx, I, _p(snr), _p(alpha))
    if rc:
        raise OracleError("noise source with zero power")
    return alpha


def mix_direct(x_sources, rirs, L, alpha, lib=None):
    """Eq. 2 for one utterance.  x_sources [I, Nx]; rirs: list of I*J arrays in
    (i, j) order; L: kept lengths [I*J]; alpha [I].  Returns y [J, Nx]."""
    x = _f64(x_sources)
    I, nx = x.shape
    J = len(rirs) // I
    off = _i64(np.concatenate([[0], np.cumsum([len(r) for r in rirs])])[:-1])
    rir = _f64(np.concatenate([np.asarray(r, dtype=np.float64) for r in rirs]))
    y = np.zeros((J, nx))
    (lib or _load()).oracle_mix_direct(_p(x), nx, I, J, _p(rir), _p(off), _p(_i64(L)),
                                       _p(_f64(alpha)), _p(y))
    return y


def mix_window(x_sources, rirs, L, alpha, n0, n1, lib=None):
    """Eq. 2 for one utterance at output positions [n0, n1) only (positions past
    Nx are those of the full output).  Arguments as mix_direct; returns [J, n1-n0]."""
    x = _f64(x_sources)
    I, nx = x.shape
    J = len(rirs) // I
    off = _i64(np.concatenate([[0], np.cumsum([len(r) for r in rirs])])[:-1])
    rir = _f64(np.concatenate([np.asarray(r, dtype=np.float64) for r in rirs]))
    y = np.zeros((J, n1 - n0))
    (lib or _load()).oracle_mix_window(_p(x), nx, I, J, _p(rir), _p(off), _p(_i64(L)), _p(_f64(alpha)),
                                       int(n0), int(n1), _p(y))
    return y


def dx_window(g_mics, rirs, L, i, alpha_i, m0, m1, lib=None):
    """Gradient of source i of one utterance at input positions [m0, m1) only.
    g_mics [J, Ny]: upstream gradient per mic; rirs, L as mix_direct."""
    g = _f64(g_mics)
    J, ny = g.shape
    off = _i64(np.concatenate([[0], np.cumsum([len(r) for r in rirs])])[:-1])
    rir = _f64(np.concatenate([np.asarray(r, dtype=np.float64) for r in rirs]))
    dx = np.zeros(m1 - m0)
    (lib or _load()).oracle_dx_window(_p(g), ny, J, int(i), _p(rir), _p(off), _p(_i64(L)), float(alpha_i),
                                      int(m0), int(m1), _p(dx))
    return dx


def dh_window(x_i, g_j, L_ij, alpha_i, k0, k1, lib=None):
    """Gradient of one RIR at taps [k0, k1): dh[k] = alpha_i sum_n g_j[n] x_i[n - k]
    for k < L_ij, 0 beyond (x_i [Nx], g_j [Ny], any Ny)."""
    x = _f64(x_i)
    g = _f64(g_j)
    out = np.zeros(int(k1) - int(k0))
    (lib or _load()).oracle_dh_window(_p(x), x.shape[0], _p(g), g.shape[0], int(L_ij), float(alpha_i),
                                      int(k0), int(k1), _p(out))
    return out


def mix_ola(x_sources, rirs, L, alpha, fft_n=0, lib=None):
    """The paper's per-(i, j) OLA filtering, FP64.  Same arguments as mix_direct."""
    x = _f64(x_sources)
    I, nx = x.shape
    J = len(rirs) // I
    off = _i64(np.concatenate([[0], np.cumsum([len(r) for r in rirs])])[:-1])
    rir = _f64(np.concatenate([np.asarray(r, dtype=np.float64) for r in rirs]))
    y = np.zeros((J, nx))
    rc = (lib or _load()).oracle_mix_ola(_p(x), nx, I, J, _p(rir), _p(off), _p(_i64(L)),
                                         _p(_f64(alpha)), int(fft_n), _p(y))
    if rc:
        raise OracleError("invalid FFT size")
    return y


def dft_real(x, n_fft, lib=None):
    x = _f64(x)
    re, im = np.zeros(n_fft), np.zeros(n_fft)
    (lib or _load()).oracle_dft_real(_p(x), x.shape[0], n_fft, _p(re), _p(im))
    return re + 1j * im


# ---- batch entry points ------------------------------------------------------
def truncate_batch(batch, eta_db, nthreads=0, lib=None):
    """Returns dict(L, peak, e_tot, e_kept) over all RIRs of the batch."""
    lib = lib or _load()
    R = batch.rir_len.shape[0]
    L = np.zeros(R, np.int64)
    pk, et, ek = np.zeros(R), np.zeros(R), np.zeros(R)
    rir = _f64(batch.rir)
    rc = lib.oracle_truncate_batch(R, _p(_i32(batch.rir_len)), _p(rir), float(eta_db),
                                   _p(L), _p(pk), _p(et), _p(ek), nthreads)
    if rc:
        raise OracleError("invalid truncation arguments")
    return dict(L=L, peak=pk, e_tot=et, e_kept=ek)


def output_lengths(batch, output_mode=0) -> np.ndarray:
    """Output samples per mic of each utterance: Nx ("same", output_mode 0) or
    Nx + max Nh - 1 over the utterance's RIRs (full convolution, mode 1)."""
    nx = np.asarray(batch.num_samples, dtype=np.int64)
    if not output_mode:
        return nx.copy()
    per_utt = np.asarray(batch.num_sources, dtype=np.int64) * batch.num_mics
    r0 = np.concatenate([[0], np.cumsum(per_utt)])
    nh = np.asarray(batch.rir_len, dtype=np.int64)
    return np.array([nx[u] + nh[r0[u]:r0[u + 1]].max() - 1 for u in range(len(nx))], dtype=np.int64)


def forward(batch, eta_db=20.0, alpha=None, nthreads=0, lib=None, output_mode=0):
    """Truncation, gains (from batch.snr_db unless alpha is given) and the
    direct-form mix (Eq. 2) over the output range of output_mode.
    Returns dict(y, alpha, L, e_kept_frac)."""
    lib = lib or _load()
    tr = truncate_batch(batch, eta_db, nthreads, lib)
    S = int(np.sum(batch.num_sources))
    gain_mode = 0 if alpha is None else 1
    a = np.zeros(S) if alpha is None else _f64(alpha).copy()
    y = np.zeros(int(np.sum(output_lengths(batch, output_mode))) * batch.num_mics)
    x = _f64(batch.x)
    rir = _f64(batch.rir)
    rc = lib.oracle_forward_batch(batch.num_sources.shape[0], batch.num_mics,
                                  _p(_i32(batch.num_sources)), _p(_i64(batch.num_samples)),
                                  _p(_i32(batch.rir_len)), _p(x), _p(rir), _p(tr["L"]),
                                  _p(_f64(batch.snr_db)), gain_mode, _p(a), _p(y), int(output_mode),
                                  nthreads)
    if rc:
        raise OracleError("noise source with zero power")
    frac = np.where(tr["e_tot"] > 0, tr["e_kept"] / np.where(tr["e_tot"] > 0, tr["e_tot"], 1), 1.0)
    return dict(y=y, alpha=a, L=tr["L"], e_kept_frac=frac)


def backward(batch, L, alpha, g, nthreads=0, lib=None, output_mode=0):
    """Adjoint of the mix for fixed L and alpha; g has the layout of the
    output_mode's y.  Returns dict(dx, dh, dalpha)."""
    lib = lib or _load()
    S = int(np.sum(batch.num_sources))
    dx = np.zeros(batch.x.shape[0])
    dh = np.zeros(batch.rir.shape[0])
    da = np.zeros(S)
    x = _f64(batch.x)
    rir = _f64(batch.rir)
    lib.oracle_backward_batch(batch.num_sources.shape[0], batch.num_mics,
                              _p(_i32(batch.num_sources)), _p(_i64(batch.num_samples)),
                              _p(_i32(batch.rir_len)), _p(x), _p(rir), _p(_i64(L)),
                              _p(_f64(alpha)), _p(_f64(g)), _p(dx), _p(dh), _p(da), int(output_mode),
                              nthreads)
    return dict(dx=dx, dh=dh, dalpha=da)


# ---- per-(source, microphone) gains (Eq. 2's alpha_ij) ------------------------
def _scaled_rirs(batch, alpha_rir):
    """The batch's RIRs each multiplied by its gain alpha_ij (RIR order)."""
    a = _f64(alpha_rir)
    assert a.shape[0] == batch.rir_len.shape[0]
    return _f64(batch.rir) * np.repeat(a, np.asarray(batch.rir_len, dtype=np.int64))


def forward_rir_gains(batch, alpha_rir, eta_db=20.0, nthreads=0, lib=None, output_mode=0):
    """Eq. 2 with one gain per (source, microphone): y_j = sum_i alpha_ij (hhat_ij * x_i).
    By linearity it is the per-source mix with unit gains of the RIRs scaled by
    alpha_ij; the cut-off (Eq. 7-9) is taken on the unscaled RIRs.  Returns
    dict(y, L)."""
    import dataclasses
    lib = lib or _load()
    tr = truncate_batch(batch, eta_db, nthreads, lib)
    S = int(np.sum(batch.num_sources))
    scaled = dataclasses.replace(batch, rir=_scaled_rirs(batch, alpha_rir))
    y = forward_with_lengths(scaled, tr["L"], np.ones(S), nthreads, lib, output_mode)
    return dict(y=y, L=tr["L"])


def backward_rir_gains(batch, L, alpha_rir, g, nthreads=0, lib=None, output_mode=0):
    """Adjoint of forward_rir_gains for fixed L: dx_i = sum_j alpha_ij (hhat_ij corr g_j),
    dh_ij = alpha_ij corr(g_j, x_i) (k < L_ij), dalpha_ij = <g_j, hhat_ij * x_i>
    = sum_k hhat_ij[k] corr(g_j, x_i)[k].  Returns dict(dx, dh, dalpha [R])."""
    import dataclasses
    lib = lib or _load()
    S = int(np.sum(batch.num_sources))
    a = _f64(alpha_rir)
    scaled = dataclasses.replace(batch, rir=_scaled_rirs(batch, a))
    out = backward(scaled, L, np.ones(S), g, nthreads, lib, output_mode)   # dh: corr(g_j, x_i)
    nh = np.asarray(batch.rir_len, dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(nh)])
    corr = out["dh"]
    rir = _f64(batch.rir)
    da = np.array([np.dot(rir[off[r]:off[r] + L[r]], corr[off[r]:off[r] + L[r]]) for r in range(nh.shape[0])])
    return dict(dx=out["dx"], dh=corr * np.repeat(a, nh), dalpha=da)


# ---- gains from SNRs on the reverberant signal (Eq. 2, SNR at a reference mic) ---
def reverberant_gains(batch, snr_db=None, eta_db=20.0, ref_mic=0, lib=None):
    """alpha_0 = 1, alpha_i = sqrt(P_0 / P_i 10^(-SNR_i/10)) with P_i the mean square
    over [0, Nx) of source i filtered by its (cut) RIR to microphone ref_mic, the
    reverberant signal that microphone receives from it.  Returns (alpha [S], P [S])."""
    lib = lib or _load()
    L = truncate_batch(batch, eta_db, 0, lib)["L"]
    snr = _f64(batch.snr_db if snr_db is None else snr_db)
    xo, ro, ri, si = batch.x_offsets(), batch.rir_offsets(), batch.rir_index(), batch.src_index()
    J = batch.num_mics
    P = np.zeros(int(si[-1]))
    alpha = np.zeros(int(si[-1]))
    for u in range(batch.num_utts):
        nx = int(batch.num_samples[u])
        for i in range(int(batch.num_sources[u])):
            s = int(si[u]) + i
            r = int(ri[u]) + i * J + ref_mic
            y = mix_direct(batch.x[xo[s]:xo[s + 1]].reshape(1, nx), [batch.rir[ro[r]:ro[r + 1]]], [L[r]], [1.0],
                           lib)
            P[s] = float(np.mean(y[0] ** 2))
        s0 = int(si[u])
        alpha[s0] = 1.0
        for i in range(1, int(batch.num_sources[u])):
            if not P[s0 + i] > 0:
                raise OracleError("noise source with zero reverberant power")
            alpha[s0 + i] = math.sqrt(P[s0] / P[s0 + i] * 10.0 ** (-snr[s0 + i] / 10.0))
    return alpha, P


def forward_with_lengths(batch, L, alpha, nthreads=0, lib=None, output_mode=0):
    """The direct-form mix (Eq. 2) for given kept lengths L and per-source gains."""
    lib = lib or _load()
    y = np.zeros(int(np.sum(output_lengths(batch, output_mode))) * batch.num_mics)
    a = _f64(alpha).copy()
    rc = lib.oracle_forward_batch(batch.num_sources.shape[0], batch.num_mics,
                                  _p(_i32(batch.num_sources)), _p(_i64(batch.num_samples)),
                                  _p(_i32(batch.rir_len)), _p(_f64(batch.x)), _p(_f64(batch.rir)), _p(_i64(L)),
                                  _p(np.zeros(a.shape[0])), 1, _p(a), _p(y), int(output_mode), nthreads)
    if rc:
        raise OracleError("invalid forward arguments")
    return y


def forward_ola(batch, L, alpha, fft_n=0, nthreads=0, lib=None):
    """The paper's OLA filtering over a batch (FP64), for given L and alpha."""
    lib = lib or _load()
    y = np.zeros(int(np.sum(batch.num_samples)) * batch.num_mics)
    x = _f64(batch.x)
    rir = _f64(batch.rir)
    rc = lib.oracle_forward_ola_batch(batch.num_sources.shape[0], batch.num_mics,
                                      _p(_i32(batch.num_sources)), _p(_i64(batch.num_samples)),
                                      _p(_i32(batch.rir_len)), _p(x), _p(rir), _p(_i64(L)),
                                      _p(_f64(alpha)), int(fft_n), _p(y), nthreads)
    if rc:
        raise OracleError("invalid FFT size")
    return y


# ---- Eq. 1: image-method RIRs ------------------------------------------------
def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def image_list(room, src, mic, refl, order=8, fs=16000.0, c0=343.0, lib=None):
    """Every image of one (source, microphone) pair in a room, virtual rooms in
    (a, b, c) order with c fastest.  Returns dict(pos [V, 3], g, delay, amp,
    travel): travel is d fs / c0 in samples (FP64) and delay = ceil(travel)."""
    V = (2 * int(order) + 1) ** 3
    pos, amp, travel = np.zeros((V, 3)), np.zeros(V), np.zeros(V)
    g, delay = np.zeros(V, np.int32), np.zeros(V, np.int64)
    n = (lib or _load()).oracle_image_list(_p(_f32(room)), _p(_f32(src)), _p(_f32(mic)), float(refl),
                                           int(order), float(fs), float(c0), _p(pos), _p(g), _p(delay),
                                           _p(amp), _p(travel))
    if n < 0:
        raise OracleError("invalid image-method arguments")
    return dict(pos=pos, g=g, delay=delay, amp=amp, travel=travel)


def image_rir(room, src, mic, refl, n_h, order=8, fs=16000.0, c0=343.0, lib=None):
    """Eq. 1 for one (source, microphone) pair: returns (h [n_h] FP64, images landed)."""
    h = np.zeros(int(n_h))
    n = (lib or _load()).oracle_image_rir(_p(_f32(room)), _p(_f32(src)), _p(_f32(mic)), float(refl),
                                          int(order), float(fs), float(c0), int(n_h), _p(h))
    if n < 0:
        raise OracleError("invalid image-method arguments")
    return h, int(n)


def image_rirs(geom, rir_len, order=8, fs=16000.0, c0=343.0, nthreads=0, lib=None):
    """Eq. 1 over a batch.  geom [R, 10] float32 rows (room, source, microphone,
    r); rir_len [R].  Returns (h packed FP64 [sum rir_len], valid bool [R])."""
    geom = _f32(geom).reshape(-1, 10)
    R = geom.shape[0]
    off = _i64(np.concatenate([[0], np.cumsum(np.asarray(rir_len, dtype=np.int64))]))
    h = np.zeros(int(off[-1]))
    valid = np.zeros(R, np.int32)
    (lib or _load()).oracle_image_rirs(R, _p(geom), _p(off), int(order), float(fs), float(c0), _p(h),
                                       _p(valid), nthreads)
    return h, valid.astype(bool)


# ---- Sec. 3: log-Mel front end ------------------------------------------------
# the paper's features: 32 ms windows every 10 ms at 16 kHz, 128 Mel bands over
# 125-7500 Hz, four frames stacked, every third stacked frame kept
MEL_DEFAULTS = dict(n_fft=512, hop=160, fs=16000.0, n_mels=128, f_lo=125.0, f_hi=7500.0, floor=1e-6,
                    stack=4, stride=3)


def hz_to_mel(f, lib=None):
    return (lib or _load()).oracle_hz_to_mel(float(f))


def mel_to_hz(m, lib=None):
    return (lib or _load()).oracle_mel_to_hz(float(m))


def mel_filters(n_fft=512, fs=16000.0, n_mels=128, f_lo=125.0, f_hi=7500.0, lib=None):
    """Triangular Mel filter weights [n_mels, n_fft/2 + 1]."""
    W = np.zeros((n_mels, n_fft // 2 + 1))
    (lib or _load()).oracle_mel_filters(int(n_fft), float(fs), int(n_mels), float(f_lo), float(f_hi), _p(W))
    return W


def frame_power(x, n_fft=512, lib=None):
    """|X[k]|^2, k = 0 .. n_fft/2, of one Hann-windowed frame of n_fft samples."""
    x = _f64(x)
    assert x.shape[0] >= n_fft
    P = np.zeros(n_fft // 2 + 1)
    (lib or _load()).oracle_frame_power(_p(x), int(n_fft), _p(P))
    return P


def log_mel_rows(n, n_fft=512, hop=160, stack=4, stride=3, lib=None):
    return int((lib or _load()).oracle_log_mel_rows(int(n), int(n_fft), int(hop), int(stack), int(stride)))


def log_mel(y, lib=None, **kw):
    """Stacked log-Mel features of one channel: [rows, stack * n_mels]."""
    p = dict(MEL_DEFAULTS, **kw)
    y = _f64(y)
    rows = log_mel_rows(y.shape[0], p["n_fft"], p["hop"], p["stack"], p["stride"], lib)
    out = np.zeros((rows, p["stack"] * p["n_mels"]))
    (lib or _load()).oracle_log_mel(_p(y), y.shape[0], p["n_fft"], p["hop"], p["fs"], p["n_mels"], p["f_lo"],
                                    p["f_hi"], p["floor"], p["stack"], p["stride"], _p(out))
    return out


def log_mel_batch(y, num_out, num_mics, channel=0, nthreads=0, lib=None, **kw):
    """Features of channel `channel` of every utterance of a mixed output laid
    out [sum_u J * Ny_u].  Returns (features [rows, stack * n_mels], row offsets [U + 1])."""
    p = dict(MEL_DEFAULTS, **kw)
    lib = lib or _load()
    ny = _i64(num_out)
    rows = np.array([log_mel_rows(n, p["n_fft"], p["hop"], p["stack"], p["stride"], lib) for n in ny], np.int64)
    off = _i64(np.concatenate([[0], np.cumsum(rows)]))
    out = np.zeros((int(off[-1]), p["stack"] * p["n_mels"]))
    lib.oracle_log_mel_batch(ny.shape[0], int(num_mics), _p(ny), _p(_f64(y)), int(channel), p["n_fft"], p["hop"],
                             p["fs"], p["n_mels"], p["f_lo"], p["f_hi"], p["floor"], p["stack"], p["stride"],
                             _p(off), _p(out), nthreads)
    return out, off


def eta_is_none(eta_db) -> bool:
    return math.isinf(eta_db)
