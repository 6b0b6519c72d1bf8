"""Build ``liblbm.so`` in-tree: sm_103a CUDA kernels + host C++ behind the C
ABI of ``include/lbm.h``.  Translation units compile in parallel; no cmake."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblbm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
CU_SOURCES = ["lbm_api.cu", "kernels_f64.cu", "kernels_f32.cu",
              "kernels_f16dev.cu", "lbm_batch.cu", "lbm_rwpt.cu"]
CPP_SOURCES = ["geometry.cpp"]
HEADERS = ["lbm_internal.h", "lbm_kernels.cuh", "lbm_launch_impl.cuh",
           "lbm_f16.cuh", "lbm_nvtx.h", "lbm_adjoint.cuh"]


def _cu_cmd(src, obj):
    return [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-c",
            "-Xcompiler", "-fPIC,-ffp-contract=off", "-Xptxas", "-v",
            os.path.join(CSRC, src), "-o", obj]


def _cpp_cmd(src, obj):
    return ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-c",
            os.path.join(CSRC, src), "-o", obj]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [
        os.path.join(HERE, "..", "include", "lbm.h")]
    jobs = []
    objs = []
    for src in CU_SOURCES + CPP_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        if force or _stale(obj, [os.path.join(CSRC, src)] + hdrs):
            cmd = _cu_cmd(src, obj) if src.endswith(".cu") else _cpp_cmd(src, obj)
            log = open(obj + ".log", "w")
            jobs.append((src, subprocess.Popen(cmd, stdout=log,
                                               stderr=subprocess.STDOUT), log))
    failed = []
    for src, proc, log in jobs:
        rc = proc.wait()
        log.close()
        if rc != 0 or verbose:
            with open(log.name) as fh:
                sys.stderr.write(fh.read())
        if rc != 0:
            failed.append(src)
    if failed:
        raise RuntimeError(f"liblbm build failed: {failed}")
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs], check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
