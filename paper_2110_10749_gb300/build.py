"""Build libssd.so (CUDA, sm_103a) in-tree: paper_2110_10749_gb300/_build/.

The translation units compile in parallel with nvcc and link into one
shared library with the CUDA runtime linked statically.  Usage:
    python -m paper_2110_10749_gb300.build [--force]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libssd.so")
SOURCES = ["ctx.cu", "pair.cu", "quad.cu", "solve.cu", "batch.cu", "geom.cu", "field.cu"]
HEADERS = ["internal.h", "series_coef.h", "erfcx_coef.h", os.path.join("..", "..", "include", "ssd.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS_EXTRA = []
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "--expt-relaxed-constexpr"]
# quadrature points are reproducible bit for bit only without FMA contraction
FILE_FLAGS = {"quad.cu": ["--fmad=false"]}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    FLAGS_EXTRA.clear()
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *FILE_FLAGS.get(src, []), *FLAGS_EXTRA, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        return obj, r.stdout + r.stderr

    # tile-shape overrides for tuning sweeps (see csrc/internal.h)
    for key in ("SSD_TPB32", "SSD_MINCTA32", "SSD_TPT32", "SSD_SYMTPT", "SSD_SYMMINCTA"):
        if os.environ.get(key):
            FLAGS_EXTRA.append("-D%s=%d" % (key, int(os.environ[key])))
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            sys.stdout.write(log)
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
