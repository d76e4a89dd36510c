"""Build the in-tree CUDA library ``libptt.so`` for sm_103a with nvcc.

Five translation units compiled in parallel, linked with the static CUDA
runtime.  Usage: ``python -m paper_2606_09468_gb300.build`` or ``build()``."""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libptt.so")
SOURCES = ["ptt_kernels.cu", "ptt_kernels3d.cu", "ptt_capi.cu", "ptt_noalloc.cu", "ptt_mma.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(verbose=False, extra=()):
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    objs = [os.path.join(OUT, s.replace(".cu", ".o")) for s in SOURCES]
    cmds = [[nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, s), "-o", o]
            for s, o in zip(SOURCES, objs)]
    with cf.ThreadPoolExecutor(len(cmds)) as ex:
        logs = list(ex.map(_run, cmds))
    logs.append(_run([nvcc, *ARCH, "-shared", "-cudart", "static", "-Xlinker", "--no-undefined",
                      "-o", LIB, *objs]))
    if verbose:
        for lg in logs:
            if lg.strip():
                print(lg)
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv, extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
    print(LIB)
