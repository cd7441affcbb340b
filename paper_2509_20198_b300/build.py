"""Build of liblidarscout.so (nvcc, sm_103a) in-tree, next to this file."""
from __future__ import annotations

import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "liblidarscout.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _stale(target, sources):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/liblidarscout.cu (which includes every source) to liblidarscout.so."""
    sources = (glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
               + glob.glob(os.path.join(INCLUDE, "*.h")))
    if force or _stale(LIB, sources):
        cmd = [NVCC, *ARCH, "-O3", "-std=c++17", "-lineinfo", "--use_fast_math",
               "-Xcompiler", "-fPIC,-O2", "-shared", "-I", INCLUDE,
               "-o", LIB + ".tmp", os.path.join(CSRC, "liblidarscout.cu")]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.check_call(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


def build_synth(force: bool = False) -> str:
    """Compile the seeded GPU input generator (synth/synth_gpu.cu) to synth/libsynth.so."""
    src = os.path.join(ROOT, "synth", "synth_gpu.cu")
    out = os.path.join(ROOT, "synth", "libsynth.so")
    if force or _stale(out, [src]):
        subprocess.check_call([NVCC, *ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                               "-shared", "-o", out + ".tmp", src])
        os.replace(out + ".tmp", out)
    return out


if __name__ == "__main__":
    print(build_library(force=True, verbose=True))
    print(build_synth(force=True))
