"""Compile the CUDA/C++ sources of the package into an in-tree shared library.

nvcc for sm_103a only (`-gencode arch=compute_103a,code=sm_103a`), g++ for the
host planner; translation units are compiled in parallel.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libcasimir.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU = ["step2d.cu", "step2d_t2.cu", "step2d_tk.cu", "step6.cu", "step6m.cu", "step6x.cu", "step6c2.cu", "step6m2.cu", "step3c.cu",
      "engine.cu", "plain.cu"]
CXX = ["plan.cpp"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def sources():
    return [os.path.join(CSRC, f) for f in CU + CXX] + [
        os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))] + [os.path.join(ROOT, "include", "casimir.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force: bool = False, verbose: bool = False, defines=()) -> str:
    """defines: extra -D macros for the CUDA sources (tuning constants); a build with them is
    always fresh."""
    if not force and not defines and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    nvcc = _nvcc()
    jobs = []
    objs = []
    for f in CU:
        o = os.path.join(OUT_DIR, f + ".o")
        objs.append(o)
        cmd = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", *inc,
               *["-D" + d for d in defines], "-c", os.path.join(CSRC, f), "-o", o]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append(cmd)
    for f in CXX:
        o = os.path.join(OUT_DIR, f + ".o")
        objs.append(o)
        jobs.append(["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", *inc, "-I", "/usr/local/cuda/include",
                     "-c", os.path.join(CSRC, f), "-o", o])
    procs = [subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for j in jobs]
    failed = []
    for j, p in zip(jobs, procs):
        out = p.communicate()[0].decode(errors="replace")
        if p.returncode != 0:
            failed.append((j, out))
        elif verbose and out.strip():
            sys.stderr.write(out)
    if failed:
        msg = "\n".join(" ".join(j) + "\n" + out for j, out in failed)
        raise RuntimeError("build failed:\n" + msg)
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
