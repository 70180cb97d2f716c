"""Build the in-tree CUDA library ``_lib/libmatex.so`` for sm_103a.

Each translation unit is compiled in parallel (nvcc for .cu, g++ for the host
setup .cpp), then linked into one shared library exposing the C ABI of
``include/matex.h``.  Rebuilds only when a source or header is newer than the
library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libmatex.so")
GENCODE = "arch=compute_103a,code=sm_103a"


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    hdr = sorted(f for f in os.listdir(CSRC) if f.endswith((".h", ".cuh")))
    return cu, cpp, hdr


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmatex")
    return cand


def _needs_build():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    cu, cpp, hdr = _sources()
    files = [os.path.join(CSRC, f) for f in cu + cpp + hdr]
    files += [os.path.join(ROOT, "include", "matex.h"), os.path.abspath(__file__)]
    return any(os.path.getmtime(f) > t for f in files)


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + p.stdout)
    return p.stdout


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and not _needs_build():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    cu, cpp, _ = _sources()
    jobs = []
    for f in cu:
        obj = os.path.join(OUT, f[:-3] + ".o")
        cmd = [nvcc, "-gencode", GENCODE, "-O3", "-lineinfo", "-std=c++17",
               "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-c",
               os.path.join(CSRC, f), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((cmd, obj))
    for f in cpp:
        obj = os.path.join(OUT, f[:-4] + ".o")
        cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-pthread", "-I", os.path.join(ROOT, "include"),
               "-c", os.path.join(CSRC, f), "-o", obj]
        jobs.append((cmd, obj))
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        outs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose or ptxas_info:
        for o in outs:
            if o.strip():
                print(o)
    objs = [o for _, o in jobs]
    tmp = LIB + ".tmp"
    # --no-undefined: a declared but missing function fails here, not at load time
    _run([nvcc, "-shared", "-gencode", GENCODE, "-o", tmp] + objs +
         ["-lcudart", "-lpthread", "-Xlinker", "--no-undefined"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
