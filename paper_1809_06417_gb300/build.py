"""Builds libflamerec.so (the C-ABI library) for sm_103a with nvcc.

Each translation unit compiles in parallel; the library links against the
static CUDA runtime so it loads on hosts without a GPU driver (there it only
exports symbols; every call needs a GPU).
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libflamerec.so")
# the checked build (bounds checks recorded in a device word): its own objects and library
LIB_CHECKED = os.path.join(BUILD, "checked", "libflamerec_checked.so")
SOURCES = ["march.cu", "volume.cu", "api.cu", "server.cu", "tables.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _flags(extra=()):
    # FR_NVCC_FLAGS: extra nvcc options (e.g. -DFR_MARCH_MINB=6 to cap march registers)
    user = os.environ.get("FR_NVCC_FLAGS", "").split()
    # -ftz=true: single-precision denormals flush to zero (no denormal paths
    # around the exp / rsqrt of the marches)
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-ftz=true", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                   "-I", CSRC, *user, *extra]


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "flamerec.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def _stamp(out_dir) -> str:
    return os.path.join(out_dir, "flags.txt")


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, checked: bool = False) -> str:
    """Compiles the library (checked: the bounds-checked variant, LIB_CHECKED)."""
    flags = os.environ.get("FR_NVCC_FLAGS", "")
    out_dir = os.path.join(BUILD, "checked") if checked else BUILD
    lib = LIB_CHECKED if checked else LIB
    same_flags = os.path.exists(_stamp(out_dir)) and open(_stamp(out_dir)).read() == flags
    if not force and same_flags and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + (["-DFR_CHECKED"] if checked else [])

    def compile_one(src):
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        cmd = [cc, *_flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose or ptxas_info:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [cc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-cudart", "static", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(_stamp(out_dir), "w") as f:
        f.write(flags)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                checked="--checked" in sys.argv))
