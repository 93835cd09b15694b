"""In-tree build of libcollage.so for sm_103a (nvcc, one process per translation unit).

Two variants from the same sources: libcollage.so, and libcollage_checked.so compiled with
-DCOLLAGE_CHECKED (index checks that latch an error bit instead of accessing past a bound, and
NVTX ranges around every kernel launch of an iteration)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libcollage.so")
LIB_CHECKED = os.path.join(OUT_DIR, "libcollage_checked.so")
SOURCES = ["api.cu", "bin.cu", "raster.cu", "loss.cu", "fit.cu", "mat.cu", "metrics.cu", "noalloc.cu", "peak.cu", "sched.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
         "-I" + INCLUDE, "-I" + CSRC]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps():
    return [os.path.join(CSRC, s) for s in SOURCES] + [
        os.path.join(CSRC, "internal.h"), os.path.join(INCLUDE, "collage.h")]


def _fresh(lib):
    return os.path.exists(lib) and all(os.path.getmtime(d) <= os.path.getmtime(lib) for d in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit of both variants (in parallel) and link libcollage.so and
    libcollage_checked.so; returns the path of libcollage.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and _fresh(LIB) and _fresh(LIB_CHECKED):
        return LIB
    nvcc = _nvcc()
    jobs = []
    for tag, extra in (("", []), ("_checked", ["-DCOLLAGE_CHECKED"])):
        for src in SOURCES:
            jobs.append((src, os.path.join(OUT_DIR, src.replace(".cu", tag + ".o")), extra))

    def compile_one(job):
        src, obj, extra = job
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src} {extra}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout, r.stderr)

    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        list(ex.map(compile_one, jobs))
    for lib, tag in ((LIB, ""), (LIB_CHECKED, "_checked")):
        objs = [os.path.join(OUT_DIR, src.replace(".cu", tag + ".o")) for src in SOURCES]
        tmp = lib + f".tmp{os.getpid()}"
        r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
