"""Build step of the package: compiles csrc/*.cu for sm_103a with nvcc and
links them into paper_2212_02988_gb300/libprism.so (in-tree), and the same
sources with -DPRISM_CHECKED into libprism_checked.so (the bounds-check
build, prism_check_status in include/prism.h).

    python -m paper_2212_02988_gb300.build [--force] [--checked-only | --no-checked]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libprism.so")
OUT_DIR_CHECKED = os.path.join(PKG, "_build_checked")
LIB_CHECKED = os.path.join(PKG, "libprism_checked.so")
SOURCES = ["render.cu", "track.cu", "state.cu", "fuse.cu", "mapio.cu", "prism_abi.cu", "noalloc.cu",
           "render_bwd.cu", "serve_kernels.cu", "serve.cu", "adam.cu", "rollout.cu", "mapping.cu"]
HEADERS = ["prism_dev.cuh", "linalg64.cuh", "kernels.h", "render_dev.cuh", "track_dev.cuh", "fuse_dev.cuh",
           "state_dev.cuh", "serve.h", "host_util.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: device code contracts no multiply-add on its own, so every
# value is the rounding sequence its source spells out (fused operations are
# written as fma / fmaf / intrinsics where wanted) whatever kernel a shared
# device body is inlined into; host code likewise with -ffp-contract=off.
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC,-ffp-contract=off",
              "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", h)
                                                        for h in ("prism.h", "prism_serve.h")]
    return max(os.path.getmtime(f) for f in files)


def _compile(src: str, force: bool, verbose: bool, checked: bool = False) -> str:
    obj = os.path.join(OUT_DIR_CHECKED if checked else OUT_DIR, src.replace(".cu", ".o"))
    s = os.path.join(CSRC, src)
    if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(s), _deps_mtime()):
        return obj
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *(["-DPRISM_CHECKED"] if checked else []), "-c", s, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        sys.stderr.write(r.stderr)
    return obj


def _link(lib: str, objs: list, force: bool) -> None:
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs):
        tmp = lib + f".tmp{os.getpid()}"
        r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False, checked: bool = True, plain: bool = True) -> str:
    """Compile (in parallel) and link libprism.so and, with `checked`, the
    bounds-check build libprism_checked.so; returns libprism.so's path."""
    jobs = ([False] if plain else []) + ([True] if checked else [])
    for c in jobs:
        os.makedirs(OUT_DIR_CHECKED if c else OUT_DIR, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES) * len(jobs)) as ex:
        objs = {c: list(ex.map(lambda s, c=c: _compile(s, force, verbose, c), SOURCES)) for c in jobs}
    for c in jobs:
        _link(LIB_CHECKED if c else LIB, objs[c], force)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--no-checked" not in sys.argv,
                plain="--checked-only" not in sys.argv))
