"""Build liblbm.so (the C-ABI library) in-tree with nvcc for sm_103a.

Translation units: api.cu (C ABI, scheduler), plan.cpp (host list builder, OpenMP), diag.cu,
reduce_static.cu, closure.cu (closure sweep and network kernels, D3Q19 FP32), halo.cu (halo
pack/unpack of partitioned runs), refine.cu (transfers of the 2:1 refinement), sweep.cu / aux.cu / sweep_sparse.cu (the fluid-cell list
sweep) compiled once per (stencil, storage) variant, sweep.cu once more per (stencil, FP64/FP32) with the MRT
collision and per FP64/FP32 D3Q27 with the cumulant collision.  Objects are compiled in parallel; the library lands in ``paper_1909_13772_gb300/_build/liblbm.so``.
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
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp", "-I", INCLUDE, "-I", CSRC,
           "--expt-relaxed-constexpr", "-Xptxas", "-O3"]
VARIANTS = [(q, st) for q in (19, 27) for st in (0, 1, 2, 3)]
MRT_VARIANTS = [(q, st) for q in (19, 27) for st in (0, 1)]  # MRT sweeps: FP64 and FP32 storage
CUM_VARIANTS = [(27, 0), (27, 1)]  # cumulant sweeps: D3Q27, FP64 and FP32 storage


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm.so")


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))] + [os.path.join(INCLUDE, "lbm.h")]


def _jobs(nvcc, extra, build_dir):
    jobs = []
    for name in ("api.cu", "plan.cpp", "diag.cu", "reduce_static.cu", "closure.cu", "halo.cu", "refine.cu"):
        src = os.path.join(CSRC, name)
        obj = os.path.join(build_dir, name.replace(".", "_") + ".o")
        lang = [] if name.endswith(".cu") else ["-x", "cu"]
        jobs.append([nvcc] + ARCH + NVFLAGS + extra + lang + ["-c", src, "-o", obj])
    for q, st in VARIANTS:
        for name in ("sweep.cu", "aux.cu", "sweep_sparse.cu"):
            src = os.path.join(CSRC, name)
            obj = os.path.join(build_dir, "%s_%d_%d.o" % (name[:-3], q, st))
            jobs.append([nvcc] + ARCH + NVFLAGS + extra + ["-DLBM_Q=%d" % q, "-DLBM_ST=%d" % st, "-c", src, "-o", obj])
    for q, st in MRT_VARIANTS:
        src = os.path.join(CSRC, "sweep.cu")
        obj = os.path.join(build_dir, "sweep_mrt_%d_%d.o" % (q, st))
        jobs.append([nvcc] + ARCH + NVFLAGS + extra + ["-DLBM_Q=%d" % q, "-DLBM_ST=%d" % st, "-DLBM_MRT_SWEEP=1", "-c", src,
                                                     "-o", obj])
    for q, st in CUM_VARIANTS:
        src = os.path.join(CSRC, "sweep.cu")
        obj = os.path.join(build_dir, "sweep_cum_%d_%d.o" % (q, st))
        jobs.append([nvcc] + ARCH + NVFLAGS + extra + ["-DLBM_Q=%d" % q, "-DLBM_ST=%d" % st, "-DLBM_CUMULANT_SWEEP=1",
                                                     "-c", src, "-o", obj])
    return jobs


def build(force: bool = False, verbose: bool = False, extra_flags=None, build_dir=None) -> str:
    """Compile (if stale) and return the path of liblbm.so.  ``extra_flags`` (e.g. -D knobs)
    and ``build_dir`` build a separate copy of the library elsewhere."""
    srcs = _sources()
    bdir = build_dir or BUILD
    lib = os.path.join(bdir, "liblbm.so")
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= max(os.path.getmtime(s) for s in srcs)):
        return lib
    nvcc = _nvcc()
    os.makedirs(bdir, exist_ok=True)
    extra = list(extra_flags or [])
    jobs = _jobs(nvcc, extra, bdir)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    workers = max(1, min(len(jobs), os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(run, jobs))
    errors = [(c, r) for c, r in results if r.returncode != 0]
    for c, r in results:
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
    if errors:
        c, r = errors[0]
        raise RuntimeError("nvcc failed:\n%s\n%s%s" % (" ".join(c), r.stdout, r.stderr))
    objs = [j[j.index("-o") + 1] for j in jobs]
    tmp = lib + ".%d.tmp" % os.getpid()
    link = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-Xcompiler", "-fopenmp", "-lgomp"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s%s" % (" ".join(link), r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import time
    t = time.time()
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
    print("%.1f s" % (time.time() - t))
