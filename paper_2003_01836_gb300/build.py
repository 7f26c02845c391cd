"""Builds libbltc.so in-tree for sm_103a with nvcc (no torch extension machinery).

Each .cu file is compiled in parallel, then linked into one shared library exporting the
C ABI of include/bltc.h.  The files that decide the tree and the lists are compiled with
--fmad=false so that their FP64 arithmetic is never contracted into fused multiply-adds.
"""
from __future__ import annotations

import concurrent.futures as cf
import fcntl
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libbltc.so")

SOURCES = ["api.cu", "scan.cu", "tree.cu", "lists.cu", "upward.cu", "plan.cu", "sweep.cu", "multisweep.cu", "direct.cu",
           "server.cu", "user_kernel.cu", "cp.cu", "hermite.cu", "graph.cu"]
# the sweep device code, embedded as text for run-time compilation of user kernels
EMBED = ("sweep_device.cuh", "kSweepDeviceSource")
NO_FMAD = {"tree.cu", "lists.cu"}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbltc.so")


def _flags(src: str):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler",
                "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if src in NO_FMAD:
        f.append("--fmad=false")
    if os.environ.get("BLTC_PTXAS_VERBOSE"):
        f += ["-Xptxas", "-v"]
    return f


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in os.listdir(CSRC)] + [os.path.join(INCLUDE, "bltc.h"),
                                                                  os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    # one build at a time (ranks of a multi-process launch share the in-tree build folder)
    with open(os.path.join(BUILD, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            if not force and not _stale():
                return LIB
            return _build(verbose)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _build(verbose: bool) -> str:
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(src)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    def embed():
        text = open(os.path.join(CSRC, EMBED[0])).read()
        assert ")BLTCSRC" not in text
        gen = os.path.join(BUILD, "embedded_sources.cpp")
        with open(gen, "w") as f:
            f.write("// generated by build.py from csrc/%s\n" % EMBED[0])
            f.write("namespace bltc {\nextern const char* const %s;\n" % EMBED[1])
            f.write('const char* const %s = R"BLTCSRC(%s)BLTCSRC";\n}\n' % (EMBED[1], text))
        obj = os.path.join(BUILD, "embedded_sources.o")
        r = subprocess.run([cc, "-c", gen, "-o", obj, "-Xcompiler", "-fPIC"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"embedding failed:\n{r.stdout}\n{r.stderr}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES) + 1, os.cpu_count() or 4)) as ex:
        fut = ex.submit(embed)
        objs = list(ex.map(compile_one, SOURCES))
        objs.append(fut.result())
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
