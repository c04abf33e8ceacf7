"""Build the CUDA library ``libclbm.so`` in-tree for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel) with
``-gencode arch=compute_103a,code=sm_103a``; the objects are linked into a
shared library next to this file (``_lib/libclbm.so``).  No CPU fallback is
built: the library is the only compute path.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
SOURCES = ["clbm_batch_fp32.cu", "clbm_batch_fp16.cu", "clbm_batch_bf16.cu", "clbm_batch_fp64.cu",
           "clbm_step_fp32.cu", "clbm_step_fp16.cu", "clbm_step_bf16.cu", "clbm_step_fp64.cu",
           "clbm_step_fp16sr.cu", "clbm_step_bf16sr.cu",
           "clbm_kernels.cu", "clbm_reduce.cu", "clbm_api.cu", "clbm_batch.cu",
           "clbm_noalloc.cu", "clbm_micro.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    path = shutil.which("nvcc")
    if path:
        return path
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def library_path() -> str:
    return os.path.join(OUT_DIR, "libclbm.so")


def _flags(extra=()):
    return ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
            "--expt-relaxed-constexpr", *extra]


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc(), *_flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for obj, log in ex.map(compile_one, SOURCES):
            objs.append(obj)
            if verbose or ptxas_info:
                print(log)
    tmp = library_path() + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl",
           "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr)
    os.replace(tmp, library_path())
    return library_path()


if __name__ == "__main__":
    import sys
    print(build(verbose=True, ptxas_info="-v" in sys.argv))
