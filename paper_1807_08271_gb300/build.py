"""Build the in-tree CUDA library ``librgbid.so`` for sm_103a with nvcc.

Each translation unit under ``csrc/`` is compiled in parallel to an object
file (``-gencode arch=compute_103a,code=sm_103a -lineinfo -O3``) and the
objects are linked into ``paper_1807_08271_gb300/librgbid.so``.  A rebuild is
skipped when the library is newer than every source and header.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "librgbid.so")
# the bounds-checked variant (every gathered plane index checked and counted, see
# rgbid_debug_bounds_violations); a test build, not the product library
BUILD_CHECKED = os.path.join(PKG, "_build_checked")
LIB_CHECKED = os.path.join(PKG, "librgbid_checked.so")
# the phase-stamped variant (the split kernel records when each phase of an iteration
# ends, see rgbid_debug_phase_stamps); a diagnostic build, not the product library
BUILD_PHASES = os.path.join(PKG, "_build_phases")
LIB_PHASES = os.path.join(PKG, "librgbid_phases.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librgbid")


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def _compile(src: str, extra: list[str], build_dir: str = BUILD) -> str:
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if "-v" in extra and r.stderr:
        print(r.stderr, file=sys.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, checked: bool = False,
          phases: bool = False) -> str:
    """Compile librgbid.so (checked=True: librgbid_checked.so with -DRGBID_BOUNDS_CHECK;
    phases=True: librgbid_phases.so with -DRGBID_PHASE_STAMPS) if needed and return its path."""
    if checked and phases:
        raise ValueError("one variant at a time")
    lib, build_dir = (LIB_CHECKED, BUILD_CHECKED) if checked else ((LIB_PHASES, BUILD_PHASES) if phases else (LIB, BUILD))
    if not force and up_to_date(lib):
        return lib
    os.makedirs(build_dir, exist_ok=True)
    extra = list(extra or []) + (["-DRGBID_BOUNDS_CHECK"] if checked else []) + \
        (["-DRGBID_PHASE_STAMPS"] if phases else [])
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(sources()), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, build_dir), sources()))
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}", file=sys.stderr)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None)
