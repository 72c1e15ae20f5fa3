"""Build the native library libricmrcc.so for sm_103a (in-tree).

Compiles the CUDA sources in parallel with nvcc and links them into
paper_2511_03567_gb300/_build/libricmrcc.so.  The generated term tables
(csrc/ric_terms.inc) are committed; regenerate them with
`python -m paper_2511_03567_gb300.gen.emit` after changing the generator.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
SOURCES = ["api.cu", "batch.cu", "planner.cu", "kernels.cu", "noalloc.cu", "tcgemm.cu", "grouped.cu", "schedule.cu", "ladder.cu", "ozaki.cu"]
HOST_SOURCES = ["full_terms.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"]
LIBNAME = "libricmrcc.so"


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _newer(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def cuda_include():
    return os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


def unpack_full_terms(force=False):
    """csrc/ric_terms_full.inc.gz -> _build/ric_terms_full.inc (when newer)."""
    import gzip
    src = os.path.join(CSRC, "ric_terms_full.inc.gz")
    dst = os.path.join(OUT, "ric_terms_full.inc")
    if force or _newer(dst, [src]):
        with gzip.open(src, "rb") as f, open(dst + ".tmp", "wb") as g:
            g.write(f.read())
        os.replace(dst + ".tmp", dst)
    return dst


def build(force=False, verbose=False):
    os.makedirs(OUT, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".inc"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "ricmrcc.h"))
    full_inc = unpack_full_terms(force)
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _newer(o, [s] + headers):
            jobs.append([nvcc(), *ARCH, *FLAGS, "-c", s, "-o", o])
    # the unfiltered term tables: data only, a host unit (g++ at -O0 keeps
    # the 17 MB initializer quick to compile)
    for src in HOST_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT, src.replace(".cpp", ".o"))
        objs.append(o)
        if force or _newer(o, [s, full_inc] + headers):
            jobs.append(["g++", "-O0", "-std=c++17", "-fPIC", "-I", OUT, "-I", CSRC, "-I", cuda_include(),
                         "-c", s, "-o", o])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r

    with ThreadPoolExecutor(max_workers=len(SOURCES) + len(HOST_SOURCES)) as ex:
        list(ex.map(run, jobs))
    lib = os.path.join(OUT, LIBNAME)
    if force or jobs or not os.path.exists(lib):
        run([nvcc(), *ARCH, "-shared", "-o", lib, *objs, "-lcudart"])
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
