"""Build libppm.so (the CUDA kernels and the C ABI) for sm_103a, in-tree.

build(check=True) builds the bounds-checked variant libppm_check.so
(-DPPM_BOUNDS_CHECK: index checks at the table, slab and template gathers,
reported through ppm_sync); select it with PPM_LIB_PATH."""
from __future__ import annotations

import concurrent.futures
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libppm.so")
BUILD_CHECK = os.path.join(ROOT, "_build_check")
LIB_CHECK = os.path.join(HERE, "libppm_check.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
SOURCES = ["api.cu", "lens.cu", "ring.cu", "shift_add.cu", "loglike.cu", "resp_tc.cu",
           "shift_add_bwd.cu", "ring_bwd.cu", "grad.cu", "peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-lineinfo", "-O3", "-std=c++17", "--ftz=true", "-Xcompiler", "-fPIC",
                "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, ptxas_info: bool = False, check: bool = False) -> str:
    build_dir, lib = (BUILD_CHECK, LIB_CHECK) if check else (BUILD, LIB)
    flags = FLAGS + (["-DPPM_BOUNDS_CHECK"] if check else [])
    os.makedirs(build_dir, exist_ok=True)
    headers = [os.path.join(CSRC, "ppm_internal.cuh"), os.path.join(ROOT, "include", "ppm.h")]
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if _stale(o, [s] + headers) or ptxas_info:
            cmd = [NVCC] + flags + (["-Xptxas", "-v"] if ptxas_info else []) + ["-c", s, "-o", o]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for out in ex.map(run, jobs):
            if verbose and out.strip():
                print(out)
    if _stale(lib, objs):
        tmp = lib + ".tmp%d" % os.getpid()
        run([NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(verbose=True, ptxas_info="-v" in sys.argv))
