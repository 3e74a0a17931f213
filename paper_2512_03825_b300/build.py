"""Build libpt.so (the CUDA library behind include/pt.h) in-tree for sm_103a.

nvcc cross-compiles without a GPU. The library links the CUDA runtime statically and
exports only the pt_* symbols. build(debug=True) builds libpt_debug.so instead: the same
sources compiled with PT_DEBUG, whose kernels check every index and record double writes
(pt_debug_report); it is loaded with PT_LIBRARY=debug.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpt.so")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libpt_debug.so")
SOURCES = ["pt_host.cpp", "pt_kernels.cu", "pt_batch.cu", "pt_flat.cu", "pt_persist.cu", "pt_flow.cu", "pt_flip.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-I", os.path.join(ROOT, "include"),
                   "-I", CSRC, "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                   "-Xcompiler", "-Wall", "--expt-relaxed-constexpr"]


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hs + [os.path.join(ROOT, "include", "pt.h"), os.path.abspath(__file__)]


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile every source that changed and link libpt.so (libpt_debug.so with debug=True);
    returns the library path."""
    bdir, lib_path = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    extra = ["-DPT_DEBUG"] if debug else []
    os.makedirs(bdir, exist_ok=True)
    hdrs = _headers()
    jobs = []
    objs = []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(bdir, src + ".o")
        objs.append(obj)
        if force or _stale(obj, [path] + hdrs):
            cmd = [NVCC] + _flags() + extra + ["-Xptxas", "-v", "-c", path, "-o", obj]
            jobs.append((src, cmd))

    def run(job):
        src, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, cmd, r

    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        for src, cmd, r in ex.map(run, jobs):
            with open(os.path.join(bdir, src + ".log"), "w") as f:
                f.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
    if force or jobs or _stale(lib_path, objs):
        vs = os.path.join(bdir, "exports.map")
        with open(vs, "w") as f:
            f.write("{ global: pt_*; local: *; };\n")
        tmp = lib_path + ".tmp%d" % os.getpid()
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + [
            "-Xlinker", "--version-script=" + vs, "-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
