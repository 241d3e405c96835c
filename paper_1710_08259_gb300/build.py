"""Build libsph_gb300.so in-tree with nvcc for sm_103a (GB300).

One nvcc process per translation unit, run in parallel, then a link step.
Objects go to paper_1710_08259_gb300/_build/ (git-ignored); the library to
paper_1710_08259_gb300/libsph_gb300.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsph_gb300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
              "--expt-relaxed-constexpr",
              "-Xptxas", "-warn-spills", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [
        os.path.join(ROOT, "include", "sph.h"), os.path.abspath(__file__)]


def _stale(target, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def _compile(src, extra, build_dir=BUILD):
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    hdrs = sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(ROOT, "include", "sph.h"),
                                                            os.path.abspath(__file__)]
    if not _stale(obj, [src] + hdrs):
        return obj, ""
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return obj, r.stderr


LIB_CHECK = os.path.join(HERE, "libsph_gb300_check.so")
BUILD_CHECK = os.path.join(HERE, "_build_check")


def build(force: bool = False, verbose: bool = False, extra=(), check: bool = False) -> str:
    """Compile every CUDA source of the library; return the .so path.
    check=True builds the bounds-checked flavour (-DSPH_CHECK: an index that
    would leave its buffer sets SPH_STATUS_BOUNDS and the access is skipped)
    as libsph_gb300_check.so, loaded by the package when SPH_CHECKED=1."""
    lib_path, build_dir = (LIB_CHECK, BUILD_CHECK) if check else (LIB, BUILD)
    if check:
        extra = list(extra) + ["-DSPH_CHECK"]
    os.makedirs(build_dir, exist_ok=True)
    if not force and not _stale(lib_path, _deps()):
        return lib_path
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(lambda s: _compile(s, list(extra), build_dir), srcs))
    if verbose:
        for _, log in results:
            if log:
                sys.stderr.write(log)
    objs = [o for o, _ in results]
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart=static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, check="--check" in sys.argv))
