"""Build the in-tree WQ library ``lib/libwq.so`` for sm_103a.

nvcc compiles every translation unit in parallel
(``-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo``), g++ the host set-up,
and nvcc links them into one shared library with the static CUDA runtime.
Run ``python -m paper_2605_29334_gb300.build`` or call ``build()``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(OUT_DIR, "libwq.so")
OBJ_DIR = os.path.join(HERE, "_build")

CU_SOURCES = ["api.cu", "k_eval.cu", "k_assemble.cu", "k_tile.cu", "k_tc.cu", "k_tsvd.cu", "noalloc.cu", "k_refine.cu"]
CPP_SOURCES = ["host.cpp", "refine_host.cpp"]
HEADERS = ["wq_internal.h", "dev.cuh", "kernels.h", "rule.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (set NVCC or install the CUDA toolkit)")


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(HERE, "..", "include", "wq.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(verbose=False, force=False, extra_nvcc=()):
    nvcc = _nvcc()
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(OBJ_DIR, exist_ok=True)
    jobs, objs = [], []
    for src in CU_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJ_DIR, src + ".o")
        objs.append(o)
        if force or _stale(o, s):
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-Xptxas", "-warn-spills", *extra_nvcc, "-c", s, "-o", o]
            jobs.append((cmd, src))
    for src in CPP_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJ_DIR, src + ".o")
        objs.append(o)
        if force or _stale(o, s):
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-c", s, "-o", o]
            jobs.append((cmd, src))
    procs = [(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), src, cmd) for cmd, src in jobs]
    failed = []
    for p, src, cmd in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append((src, text))
        elif verbose and text.strip():
            print("[%s]\n%s" % (src, text))
    if failed:
        msg = "\n".join("--- %s ---\n%s" % f for f in failed)
        raise RuntimeError("WQ library build failed:\n" + msg)
    if force or jobs or not os.path.exists(LIB):
        link = [nvcc, *ARCH, "-shared", "-o", LIB, *objs, "-cudart", "static"]
        r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
