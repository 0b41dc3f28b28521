"""Builds the in-tree CUDA library libholstein_dqmc.so for sm_103a (GB300).

nvcc compiles each translation unit in parallel, then links one shared library next to
this file.  Nothing is installed outside the source tree.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libholstein_dqmc.so")
SOURCES = ["hq_kernels.cu", "hq_nn.cu", "hq_cnn.cu", "hq_engine.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", os.path.join(ROOT, "include")]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False, extra=(), variant=None):
    """Compile and link the library; with `variant` (e.g. "timing" with extra=("-DHQ_SECTION_TIMING",))
    into its own build directory and libholstein_dqmc_<variant>.so, leaving the default build alone."""
    build_dir = BUILD if variant is None else BUILD + "_" + variant
    lib = LIB if variant is None else os.path.join(HERE, f"libholstein_dqmc_{variant}.so")
    os.makedirs(build_dir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "holstein_dqmc.h"))
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src.replace(".cu", ".o"))
        if _stale(o, [s] + headers):
            jobs.append([nvcc(), *ARCH, *FLAGS, *extra, "-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for out in ex.map(run, jobs):
            if verbose and out.strip():
                print(out)
    objs = [os.path.join(build_dir, s.replace(".cu", ".o")) for s in SOURCES]
    if _stale(lib, objs):
        run([nvcc(), *ARCH, "-shared", "-o", lib, *objs])
    return lib


if __name__ == "__main__":
    build(verbose=True, extra=tuple(sys.argv[1:]))
