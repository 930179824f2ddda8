"""Builds librsim.so (sm_103a) in-tree with nvcc; translation units compile in parallel."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ_DIR = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(PKG, "librsim.so")

SOURCES = ["rsim_prep.cu", "rsim_forward.cu", "rsim_backward.cu", "rsim_api.cu", "rsim_noalloc.cu",
           "rsim_image.cu", "rsim_mel.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", f"-I{INCLUDE}", f"-I{CSRC}"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _deps():
    return [os.path.join(CSRC, s) for s in SOURCES] + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(INCLUDE, "rsim.h"), __file__]


def _stale(target, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


PROBE_SRC = os.path.join(PKG, "probe", "fp32_peak.cu")
PROBE_LIB = os.path.join(PKG, "probe", "libfp32probe.so")


def build_probe(force: bool = False) -> str:
    """The FP32 FMA-throughput probe (a separate library; the benchmark's
    roofline denominator)."""
    if not force and not _stale(PROBE_LIB, [PROBE_SRC, __file__]):
        return PROBE_LIB
    tmp = PROBE_LIB + ".tmp"
    r = subprocess.run([_nvcc(), *ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                        PROBE_SRC, "-o", tmp], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for the FP32 probe:\n{r.stderr}")
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


def build(force: bool = False, verbose: bool = False, extra_flags=(), lib_path: str = LIB_PATH,
          obj_dir: str = OBJ_DIR) -> str:
    """Compiles every CUDA translation unit for sm_103a and links librsim.so."""
    deps = _deps()
    if not force and not _stale(lib_path, deps):
        return lib_path
    os.makedirs(obj_dir, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            print(log)
    objs = [o for o, _ in results]
    tmp = lib_path + ".tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


CHECKED_LIB_PATH = os.path.join(PKG, "librsim_checked.so")


def build_checked(force: bool = False) -> str:
    """The bounds-checked variant (-DRSIM_BOUNDS_CHECK): every kernel store is
    checked against its buffer's extent, an element outside latches an error
    that rsim_plan_sync_status reports, and the store is skipped.  Built beside
    librsim.so as librsim_checked.so, for debugging and tests."""
    return build(force=force, extra_flags=("-DRSIM_BOUNDS_CHECK",), lib_path=CHECKED_LIB_PATH,
                 obj_dir=os.path.join(PKG, "_build_checked"))


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
