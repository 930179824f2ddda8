"""ctypes binding of librsim.so (argument marshalling only).

The library is built in-tree by ``paper_1712_03439_gb300.build``.  Loading
fails loudly when it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "librsim.so")

RSIM_OK = 0
STATUS_NAMES = {0: "RSIM_OK", 1: "RSIM_E_INVALID", 2: "RSIM_E_UNSUPPORTED", 3: "RSIM_E_NOMEM",
                4: "RSIM_E_CUDA", 5: "RSIM_E_DEVICE", 6: "RSIM_E_STATE"}

# every symbol include/rsim.h declares
EXPORTED = ["rsim_plan", "rsim_filter_mix", "rsim_filter_mix_backward", "rsim_plan_sync_status",
            "rsim_plan_query", "rsim_plan_set_timing", "rsim_plan_stage_times",
            "rsim_plan_scratch_bytes", "rsim_plan_destroy", "rsim_source_gains_noalloc",
            "rsim_image_rirs", "rsim_plan_log_mel", "rsim_plan_log_mel_rows", "rsim_filter_mix_rooms",
            "rsim_plan_reshape", "rsim_last_error"]
STAGES = ["truncate", "power", "plan", "spectrum", "forward", "fixup", "backward", "finalize"]


class RsimError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class PlanDesc(ctypes.Structure):
    _fields_ = [
        ("num_utts", ctypes.c_int32),
        ("num_mics", ctypes.c_int32),
        ("num_sources", ctypes.c_void_p),
        ("num_samples", ctypes.c_void_p),
        ("rir_len", ctypes.c_void_p),
        ("eta_db", ctypes.c_double),
        ("fft_sizes_mask", ctypes.c_int32),
        ("gain_mode", ctypes.c_int32),
        ("segment_len", ctypes.c_int64),
        ("bwd_segment_len", ctypes.c_int64),
        ("fft_cost", ctypes.c_void_p),
        ("disable_graphs", ctypes.c_int32),
        ("output_mode", ctypes.c_int32),
        ("snr_ref_mic", ctypes.c_int32),
        ("rooms", ctypes.c_int32),
        ("long_rirs", ctypes.c_int32),
        ("spectrum_cache", ctypes.c_int32),
    ]


class MelDesc(ctypes.Structure):
    _fields_ = [
        ("channel", ctypes.c_int32),
        ("hop", ctypes.c_int32),
        ("fs", ctypes.c_float),
        ("n_mels", ctypes.c_int32),
        ("f_lo", ctypes.c_float),
        ("f_hi", ctypes.c_float),
        ("log_floor", ctypes.c_float),
        ("stack", ctypes.c_int32),
        ("stride", ctypes.c_int32),
    ]


_lib = None


def load(path: str | None = None):
    """Loads librsim.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with paper_1712_03439_gb300.build.build()")
    lib = ctypes.CDLL(p)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.rsim_plan.restype = ctypes.c_int
    lib.rsim_plan.argtypes = [ctypes.POINTER(PlanDesc), ctypes.c_int, ctypes.POINTER(P)]
    lib.rsim_plan_reshape.restype = ctypes.c_int
    lib.rsim_plan_reshape.argtypes = [P, ctypes.POINTER(PlanDesc)]
    lib.rsim_filter_mix.restype = ctypes.c_int
    lib.rsim_filter_mix.argtypes = [P, P, P, P, P, P, P, P, P]
    lib.rsim_filter_mix_rooms.restype = ctypes.c_int
    lib.rsim_filter_mix_rooms.argtypes = [P, P, P, P, i32, ctypes.c_float, ctypes.c_float, P, P, P, P, P, P]
    lib.rsim_filter_mix_backward.restype = ctypes.c_int
    lib.rsim_filter_mix_backward.argtypes = [P, P, P, P, P, P, P, P]
    lib.rsim_plan_sync_status.restype = ctypes.c_int
    lib.rsim_plan_sync_status.argtypes = [P, P]
    lib.rsim_plan_query.restype = ctypes.c_int
    lib.rsim_plan_query.argtypes = [P, P, P, P, P, P]
    lib.rsim_plan_set_timing.restype = ctypes.c_int
    lib.rsim_plan_set_timing.argtypes = [P, ctypes.c_int]
    lib.rsim_plan_stage_times.restype = ctypes.c_int
    lib.rsim_plan_stage_times.argtypes = [P, P, P]
    lib.rsim_plan_scratch_bytes.restype = i64
    lib.rsim_plan_scratch_bytes.argtypes = [P]
    lib.rsim_plan_destroy.restype = None
    lib.rsim_plan_destroy.argtypes = [P]
    lib.rsim_source_gains_noalloc.restype = ctypes.c_int
    lib.rsim_source_gains_noalloc.argtypes = [P, ctypes.c_int32, P, P, P, P, P]
    lib.rsim_image_rirs.restype = ctypes.c_int
    lib.rsim_image_rirs.argtypes = [P, i32, P, P, i64, i32, ctypes.c_float, ctypes.c_float, P, P]
    lib.rsim_plan_log_mel.restype = ctypes.c_int
    lib.rsim_plan_log_mel.argtypes = [P, P, P, ctypes.POINTER(MelDesc), P]
    lib.rsim_plan_log_mel_rows.restype = ctypes.c_int
    lib.rsim_plan_log_mel_rows.argtypes = [P, ctypes.POINTER(MelDesc), P, P]
    lib.rsim_last_error.restype = ctypes.c_char_p
    lib.rsim_last_error.argtypes = []
    if path is None:
        _lib = lib
    return lib


def check(lib, status: int):
    if status != RSIM_OK:
        raise RsimError(status, lib.rsim_last_error().decode())
