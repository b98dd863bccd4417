"""Build libdgsem.so (CUDA kernels + C ABI) in-tree for sm_103a.

Each translation unit is compiled in parallel with nvcc, then linked into a
shared library next to this file.  Usage: python -m paper_2603_06267_gb300.build
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdgsem.so")
SOURCES = ["api.cu", "vol_f32.cu", "vol_f32_abc.cu", "vol_f64.cu", "vol_f64_abc.cu", "small.cu", "pml.cu", "surrogate.cu", "peak.cu",
           "hex_api.cu", "hex_kernels.cu", "hex_vol_f32.cu", "hex_vol_f64.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdgsem.so")


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, "internal.h"), os.path.join(CSRC, "vol_impl.cuh"), os.path.join(CSRC, "tables.h"),
               os.path.join(CSRC, "hex_geom.h"), os.path.join(CSRC, "hex_step.cuh"),
               os.path.join(CSRC, "hex_vol.cuh"), os.path.join(INCLUDE, "dgsem.h"), os.path.join(INCLUDE, "dghex.h"),
               os.path.join(INCLUDE, "surrogate.h")]
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                    "-I", CSRC, "-I", INCLUDE]
    if verbose:
        flags += ["-Xptxas", "-v"]
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc] + flags + ["-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    failed = []
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose and (r.stdout or r.stderr):
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                failed.append((cmd, r.stderr))
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + e for c, e in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    if force or jobs or not os.path.exists(LIB) or _stale(LIB, objs):
        cmd = [nvcc] + ARCH + ["-shared", "-o", LIB] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + " ".join(cmd) + "\n" + r.stderr)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
