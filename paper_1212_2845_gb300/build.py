"""Build the CUDA library ``_build/libvx.so`` for sm_103a with nvcc.

Each translation unit compiles in parallel; the objects link into one shared
library exporting the C ABI of ``include/vx.h``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
# VX_HOST_SANITIZE=1: host code built with AddressSanitizer and
# UndefinedBehaviorSanitizer into a separate folder (load the runtimes with
# LD_PRELOAD); device code is unchanged
SANITIZE = os.environ.get("VX_HOST_SANITIZE") == "1"
# VX_BOUNDS_CHECK=1: kernels built with bounds checks on the indices they read
# from device tables (a failed check sets a status bit and skips the access;
# vx_step returns VX_ERR_BOUNDS) into a separate folder
BOUNDS = os.environ.get("VX_BOUNDS_CHECK") == "1"
OUT = os.path.join(HERE, "_build_san" if SANITIZE else ("_build_bc" if BOUNDS else "_build"))
LIB = os.path.join(OUT, "libvx.so")
INCLUDE = os.path.join(ROOT, "include")

SOURCES = ["vx_host.cpp", "vx_api.cu", "vx_step.cu", "vx_collide.cu", "vx_io.cu", "vx_noalloc.cu", "vx_pipe.cu", "vx_resident.cu", "vx_adjoint.cu", "vx_audit.cu", "vx_dt.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         f"-I{INCLUDE}", f"-I{SRC}"]
SAN_FLAGS = (["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined", "-Xcompiler", "-fno-omit-frame-pointer", "-g"]
             if SANITIZE else [])  # one sanitizer per -Xcompiler: nvcc splits its argument on commas


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return exe


def _deps():
    return [os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(INCLUDE, "vx.h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    deps = _deps()
    if not force and not _stale(LIB, deps):
        return LIB
    exe = nvcc()

    def compile_one(src):
        obj = os.path.join(OUT, os.path.splitext(src)[0] + ".o")
        cmd = [exe, *ARCH, *FLAGS, *SAN_FLAGS, *(["-DVX_BOUNDS_CHECK"] if BOUNDS else []), "-c",
               os.path.join(SRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd[1:1] = ["-Xptxas", "-v"] if verbose else []
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            if log:
                print(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [exe, *ARCH, *SAN_FLAGS, "-shared", "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
