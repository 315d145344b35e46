"""Build the CUDA library libdim.so for sm_103a (in-tree, no cmake).

The translation units compile in parallel with nvcc and link into one
shared library next to this file.  Used by ``__graft_entry__.build()`` and by
the tests; nothing here runs on the GPU.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libdim.so")
SOURCES = ["dim_api.cu", "dim_sweep.cu", "dim_parabolic.cu", "dim_noalloc.cu", "dim_bulkff.cu", "dim_batch.cu",
           "dim_adjoint.cu", "dim_grad.cu", "dim_probe.cu"]
# the FP32-bulk kernels may contract multiply-adds (no bit-compatibility claim;
# their float-float operations are explicit round-to-nearest intrinsics, which
# are never contracted)
FMA_SOURCES = {"dim_bulkff.cu", "dim_batch.cu"}
HEADERS = ["dim_device.cuh", "dim_ff.cuh", "dim_ctx.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _flags():
    # --fmad=false: the FP64 kernels round every operation as written (no FMA
    # contraction), which keeps them bit-compatible with a plain IEEE-754
    # evaluation of the same formulas
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC",
                   "-I", os.path.join(ROOT, "include")]


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compile (if stale) and return the path of libdim.so."""
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", h) for h in ("dim.h", "dim_probe.h")]
    procs, objs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            flags = _flags()
            if src in FMA_SOURCES:
                flags = [f for f in flags if f != "--fmad=false"] + ["--fmad=true"]
            cmd = [NVCC] + flags + list(extra) + ["-c", s, "-o", o]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            sys.stderr.write(out.decode())
        if p.returncode:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
    if force or procs or _stale(LIB, objs):
        cmd = [NVCC] + ARCH + ["-shared", "-o", LIB] + objs
        subprocess.check_call(cmd)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
