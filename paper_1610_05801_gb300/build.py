"""Build libphtl.so in-tree with nvcc for sm_103a (no torch, no cmake).

Each CUDA translation unit is compiled in parallel, then linked into a shared
library next to this file.  The CUDA runtime is linked statically, so the library
only needs the driver at run time.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libphtl.so")
SOURCES = ["api.cu", "api_programme.cu", "api_collective.cu", "track_f64.cu", "track_f32c.cu", "track_batched.cu", "track_general.cu",
           "track_general_batched.cu", "track_general_rk4.cu", "track_general_batched_f32.cu",
           "track_general_dual.cu", "track_general_dual_f32.cu",
           "track_ramp.cu", "track_collective.cu",
           "track_collective_f32.cu", "track_collective_f32_lin.cu", "batch.cu", "server.cu", "batch_static.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", f"-I{INCLUDE}", f"-I{CSRC}"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    out = [os.path.join(INCLUDE, "phtl.h"), __file__]
    for f in os.listdir(CSRC):
        out.append(os.path.join(CSRC, f))
    return out


def _stale(target, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, extra, build_dir: str = BUILD) -> str:
    obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, extra_flags=(), lib: str = LIB,
          build_dir: str = BUILD) -> str:
    """Compile and link libphtl.so; returns its path.  Rebuilds only when a source,
    header or this script is newer than the library (or force=True).  extra_flags are
    passed to every nvcc compile (e.g. -DPHTL_F64_PARTICLES_PER_THREAD=4); lib and
    build_dir place such a variant elsewhere."""
    deps = _deps()
    if not force and not _stale(lib, deps):
        return lib
    os.makedirs(build_dir, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, list(extra_flags), build_dir), SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print(f"built {lib}")
    return lib


if __name__ == "__main__":
    build(force=True, verbose=True)
