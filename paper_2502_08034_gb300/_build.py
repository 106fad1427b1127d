"""Build the CUDA library in-tree with nvcc for sm_103a (GB300).

The shared library ``librfbsoc.so`` is placed next to this file; the Python binding
(``rfb.py``) loads it from there and fails loudly if it is missing.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "librfbsoc.so")            # the solver (C ABI of include/rfb_soc.h)
SYNTH_LIB = os.path.join(HERE, "librfbsynth.so")    # potential-flow input generator
HOST_SYNTH_LIB = os.path.join(HERE, "librfbsynth_host.so")   # the same on the host CPU
TARGETS = {
    LIB: ([os.path.join(CSRC, "rfb_soc.cu")],
          # every kernel header of csrc/ and the C ABI header
          sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")) +
          [os.path.join(ROOT, "include", "rfb_soc.h")]),
    SYNTH_LIB: ([os.path.join(CSRC, "synth_flow.cu")], []),
    HOST_SYNTH_LIB: ([os.path.join(CSRC, "synth_flow_cpu.c")], []),
}
HOST_TARGETS = {HOST_SYNTH_LIB}   # plain C (gcc), no CUDA
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        p = os.path.join(cand, "bin", "nvcc") if cand else ""
        if p and os.path.exists(p):
            return p
    p = shutil.which("nvcc")
    if not p:
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librfbsoc.so")
    return p


def cuda_lib_dir() -> str:
    return os.path.join(os.path.dirname(os.path.dirname(nvcc())), "lib64")


def command(out: str = LIB, extra=(), target: str = LIB):
    sources = TARGETS[target][0]
    if target in HOST_TARGETS:
        # fixed-order sums and no contraction into FMA: the same result on every host
        return [os.environ.get("CC", "gcc"), "-O2", "-fopenmp", "-ffp-contract=off", "-shared",
                "-fPIC", *extra, "-o", out, *sources, "-lm"]
    return [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
            "-cudart", "shared", "-I", os.path.join(ROOT, "include"),
            "-Xlinker", "-rpath," + cuda_lib_dir(), *extra, "-o", out, *sources]


def up_to_date(target: str) -> bool:
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    srcs, deps = TARGETS[target]
    return all(os.path.getmtime(d) <= t for d in srcs + deps)


def _build_one(target: str, force: bool, verbose: bool):
    if not force and up_to_date(target):
        return None
    tmp = target + ".tmp"
    cmd = command(tmp, target=target)
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    return target, tmp, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                         text=True)


def build(force: bool = False, verbose: bool = False, targets=None) -> str:
    """Compile the libraries (in parallel); returns the solver library path."""
    jobs = [j for j in (_build_one(t, force, verbose) for t in (targets or TARGETS)) if j]
    errors = []
    for target, tmp, proc in jobs:
        out, err = proc.communicate()
        if proc.returncode != 0:
            errors.append("build failed for %s:\n%s%s" % (os.path.basename(target), out, err))
        else:
            os.replace(tmp, target)
    if errors:
        raise RuntimeError("\n".join(errors))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
