"""Builds libhz.so (the CUDA library behind include/hz.h) in-tree for sm_103a.

    python -m paper_2308_06152_gb300.build [-v] [--force]

Each translation unit is compiled in parallel with nvcc into ``_build/`` at
the repository root, then linked into ``paper_2308_06152_gb300/libhz.so``.
Up-to-date objects are reused.
"""

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libhz.so")
SOURCES = ["hz_stencil.cu", "hz_vcycle.cu", "hz_krylov.cu", "hz_gradient.cu",
           "hz_solver.cu", "hz_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-O2", "--expt-relaxed-constexpr"]


def _nvcc():
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build "
                       "libhz.so")


def _headers():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)
            if f.endswith((".cuh", ".h"))] + [os.path.join(INCLUDE, "hz.h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False, force=False, extra_flags=()):
    """Compile every translation unit and link libhz.so; returns its path."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    hdrs = _headers()
    jobs = []
    for src in SOURCES:
        spath = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        if force or _stale(obj, [spath] + hdrs):
            cmd = [nvcc, *ARCH, *FLAGS, *extra_flags, "-I", INCLUDE, "-I", CSRC,
                   "-c", spath, "-o", obj]
            jobs.append((src, cmd))
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in SOURCES]

    def run(job):
        src, cmd = job
        if verbose:
            print(" ".join(cmd), flush=True)
        p = subprocess.run(cmd, capture_output=True, text=True)
        return src, p.returncode, p.stdout + p.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        for src, rc, out in ex.map(run, jobs):
            if verbose and out.strip():
                print(out, flush=True)
            if rc != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{out}")
    if force or jobs or _stale(LIB, objs):
        cmd = [nvcc, *ARCH, "-shared", "-Xlinker", "--no-undefined", "-o", LIB,
               *objs]
        if verbose:
            print(" ".join(cmd), flush=True)
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("link of libhz.so failed:\n" + p.stdout + p.stderr)
    return LIB


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("-v", "--verbose", action="store_true")
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--ptxas-info", action="store_true",
                    help="print registers / spills per kernel")
    a = ap.parse_args(argv)
    extra = ("-Xptxas", "-v") if a.ptxas_info else ()
    print(build(verbose=a.verbose or a.ptxas_info, force=a.force or a.ptxas_info,
                extra_flags=extra))


if __name__ == "__main__":
    sys.exit(main())
