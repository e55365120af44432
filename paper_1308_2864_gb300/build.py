"""Compile the CUDA library (sm_103a) in-tree: csrc/*.cu -> lib/libks_gb300.so.

Each translation unit is compiled by its own nvcc process in parallel, then
linked with the static CUDA runtime, so the library only needs the driver at
run time.  Rebuilds happen when a source or header is newer than the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIBNAME = "libks_gb300.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def headers() -> list[str]:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hs


def lib_path() -> str:
    return os.path.join(LIBDIR, LIBNAME)


def mode_flags() -> list[str]:
    """Extra compiler flags of the requested build mode: KS_DEBUG_BOUNDS=1 in
    the environment selects the bounds-checked build (every checked index
    tested before its access, see ks_debug_bounds in include/ks.h)."""
    return ["-DKS_DEBUG_BOUNDS"] if os.environ.get("KS_DEBUG_BOUNDS", "0") not in ("", "0") else []


def _stamp_path() -> str:
    return os.path.join(LIBDIR, "build_flags.txt")


def needs_build() -> bool:
    out = lib_path()
    if not os.path.exists(out):
        return True
    try:
        with open(_stamp_path()) as fh:
            if fh.read().strip() != " ".join(mode_flags()):
                return True
    except OSError:
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(f) > t for f in sources() + headers() + [__file__])


def _compile(src: str, extra: list[str]) -> str:
    obj = os.path.join(OBJDIR, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Build lib/libks_gb300.so if it is missing or stale; return its path."""
    if not force and not needs_build():
        return lib_path()
    os.makedirs(OBJDIR, exist_ok=True)
    srcs = sources()
    flags = mode_flags() + list(extra or [])
    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, flags), srcs))
    tmp = lib_path() + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path())
    with open(_stamp_path(), "w") as fh:
        fh.write(" ".join(mode_flags()))
    if verbose:
        print(f"built {lib_path()}")
    return lib_path()


if __name__ == "__main__":
    build(force=True, verbose=True)
