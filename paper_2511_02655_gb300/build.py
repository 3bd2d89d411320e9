"""Builds libnbody.so (sm_103a) in-tree with nvcc: one object per .cu file,
compiled in parallel, then linked as a shared library with the shared CUDA
runtime (so that it shares the runtime instance torch has loaded).

build(debug=True) builds libnbody_debug.so instead: the same sources with
NBODY_DEBUG defined, whose kernels check every work item, chunk and system
range against the buffers it indexes (a failed check skips the access and is
reported by nbody_sync as NBODY_EINTERNAL). The binding loads it when the
environment variable NBODY_DEBUG_LIB is 1."""

from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libnbody.so")
BUILD_DIR = os.path.join(HERE, "_build")
DEBUG_LIB = os.path.join(HERE, "libnbody_debug.so")
DEBUG_BUILD_DIR = os.path.join(HERE, "_build_debug")

SOURCES = ["force_kernels.cu", "adjoint_kernels.cu", "post_kernels.cu", "capi.cu", "noalloc.cu"]
HEADERS = ["nbody_internal.h", "pair_common.cuh", "post_common.cuh", "force_common.cuh"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE,
                     "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _newer(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, debug: bool = False) -> str:
    lib_out, build_dir = (DEBUG_LIB, DEBUG_BUILD_DIR) if debug else (LIB, BUILD_DIR)
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "nbody.h")]
    flags = NVCC_FLAGS + (["-DNBODY_DEBUG"] if debug else [])
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src.replace(".cu", ".o"))
        if force or ptxas_info or _newer(o, [s] + hdrs):
            cmd = [nvcc] + flags + (["-Xptxas", "-v"] if ptxas_info else []) + ["-c", s, "-o", o]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for cmd, r in ex.map(run, jobs):
                if verbose or ptxas_info or r.returncode:
                    sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
                if r.returncode:
                    raise RuntimeError(f"nvcc failed for {cmd[-3]}")
    objs = [os.path.join(build_dir, s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or _newer(lib_out, objs):
        tmp = lib_out + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + \
              ["-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            raise RuntimeError(f"link of {os.path.basename(lib_out)} failed")
        os.replace(tmp, lib_out)
    return lib_out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                debug="--debug" in sys.argv))
