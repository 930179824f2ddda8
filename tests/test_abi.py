"""The C-ABI library builds, loads and exports every declared symbol (CPU)."""
import ctypes
import os
import re

import pytest

from paper_1712_03439_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rsim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rsim_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_header_declares_the_expected_entry_points():
    assert _declared() == sorted(_lib.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def _desc(**kw):
    import numpy as np
    ns = np.array(kw.pop("ns", [1]), np.int32)
    nx = np.array(kw.pop("nx", [100]), np.int64)
    rl = np.array(kw.pop("rl", [10]), np.int32)
    d = _lib.PlanDesc(num_utts=kw.pop("U", len(ns)), num_mics=kw.pop("J", 1),
                      num_sources=ns.ctypes.data, num_samples=nx.ctypes.data,
                      rir_len=rl.ctypes.data, eta_db=kw.pop("eta", 20.0),
                      fft_sizes_mask=kw.pop("mask", 0), gain_mode=kw.pop("gm", 0),
                      segment_len=kw.pop("seg", 0), bwd_segment_len=kw.pop("bseg", 0),
                      fft_cost=None, disable_graphs=0, output_mode=kw.pop("om", 0),
                      snr_ref_mic=kw.pop("ref", 0), rooms=kw.pop("rooms", 0),
                      long_rirs=kw.pop("long", 0), spectrum_cache=kw.pop("cache", 0))
    return d, (ns, nx, rl)


@pytest.mark.parametrize("kw,status", [
    (dict(U=0), 1),
    (dict(J=0), 1),
    (dict(eta=-1.0), 1),
    (dict(eta=float("nan")), 1),
    (dict(gm=4), 1),
    (dict(gm=-1), 1),
    (dict(gm=3, ref=1), 1),
    (dict(gm=3, ref=-1), 1),
    (dict(ns=[0]), 1),
    (dict(ns=[17], rl=[10] * 17), 1),
    (dict(nx=[0]), 1),
    (dict(rl=[0]), 1),
    (dict(mask=1 << 16), 2),
    (dict(seg=-5), 1),
    (dict(bseg=-5), 1),
    (dict(om=2), 1),
    (dict(om=-1), 1),
    (dict(rooms=2), 1),
    (dict(rooms=1, gm=3), 2),
    (dict(rooms=1, rl=[40961]), 2),
    (dict(rooms=1, eta=float("inf"), rl=[20000]), 2),
    (dict(rooms=1, long=1, rl=[20000]), 2),
    (dict(long=2), 1),
    (dict(long=-1), 1),
    (dict(cache=2), 1),
])
def test_plan_rejects_bad_descriptions_on_the_host(lib, kw, status):
    d, keep = _desc(**kw)
    h = ctypes.c_void_p()
    st = lib.rsim_plan(ctypes.byref(d), 0, ctypes.byref(h))
    assert st == status
    assert h.value is None
    assert lib.rsim_last_error().decode() != ""


def test_null_plan_calls_fail_cleanly(lib):
    assert lib.rsim_filter_mix(None, None, None, None, None, None, None, None, None) == 1
    assert lib.rsim_filter_mix_backward(None, None, None, None, None, None, None, None) == 1
    assert lib.rsim_filter_mix_rooms(None, None, None, None, 8, 16000.0, 343.0, None, None, None, None, None,
                                     None) == 1
    assert lib.rsim_plan_scratch_bytes(None) == 0
    lib.rsim_plan_destroy(None)


@pytest.mark.parametrize("args", [
    dict(R=-1),
    dict(order=-1),
    dict(order=33),
    dict(fs=0.0),
    dict(fs=float("nan")),
    dict(c0=-343.0),
    dict(c0=float("inf")),
    dict(max_len=-1),
    dict(max_len=(1 << 24) + 1),
    dict(R=2, null=True),
])
def test_image_rirs_rejects_bad_arguments_on_the_host(lib, args):
    # every case is refused before any CUDA call, so no GPU is needed
    R = args.get("R", 0)
    fake = None if args.get("null") else ctypes.c_void_p(16)
    st = lib.rsim_image_rirs(None, R, fake, fake, args.get("max_len", 100), args.get("order", 8),
                             args.get("fs", 16000.0), args.get("c0", 343.0), fake, None)
    assert st == 1
    assert "rsim_image_rirs" in lib.rsim_last_error().decode()


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes structures of the binding have the header's field offsets and sizes
    (compiled with the host C compiler against include/rsim.h)."""
    import subprocess
    structs = {"rsim_plan_desc": _lib.PlanDesc, "rsim_mel_desc": _lib.MelDesc}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "rsim.h"', 'int main(void) {']
    for cname, cls in structs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append('    printf("rsim_image_geom size %zu\\n", sizeof(rsim_image_geom));')
    lines.append('    return 0;\n}')
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, f"{cname}.{fname}"
    # the image geometry rows the binding passes: 10 floats
    assert got[("rsim_image_geom", "size")] == 40
