"""Build libsem.so in-tree: nvcc for sm_103a, one object per .cu file,
compiled in parallel, then linked with the static CUDA runtime."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsem.so")
SOURCES = ["sem_api.cu", "sem_setup.cu", "sem_ax.cu", "sem_ax32.cu", "sem_ax_lines64.cu", "sem_ax_lines32.cu",
           "sem_ax_dw.cu",
           "sem_tune.cu", "sem_cg.cu", "sem_pcg.cu", "sem_mixed.cu", "sem_batch.cu", "sem_serve.cu", "sem_probe.cu", "sem_dist.cu",
           "sem_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsem")


def _flags(verbose_ptxas: bool) -> list[str]:
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                "--expt-relaxed-constexpr"]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "sem.h"))
    cc = nvcc()
    objs, todo = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or verbose_ptxas or _stale(o, [s] + headers):
            todo.append((s, o))

    def compile_one(job):
        s, o = job
        cmd = [cc, *_flags(verbose_ptxas), "-c", s, "-o", o]
        proc = subprocess.run(cmd, capture_output=True, text=True)
        return s, proc

    if todo:
        with ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            results = list(ex.map(compile_one, todo))
        failed = [(s, p) for s, p in results if p.returncode != 0]
        for s, p in results:
            if verbose_ptxas or p.returncode != 0:
                sys.stderr.write(p.stdout + p.stderr)
        if failed:
            raise RuntimeError("nvcc failed for " + ", ".join(os.path.basename(s) for s, _ in failed))
    if force or todo or _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
        proc = subprocess.run(cmd, capture_output=True, text=True)
        if proc.returncode != 0:
            sys.stderr.write(proc.stdout + proc.stderr)
            raise RuntimeError("link of libsem.so failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
