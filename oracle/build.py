"""Build the oracle's C library (plain gcc, FP64, no FMA contraction).

TEST INFRASTRUCTURE: builds ``oracle/_build/liboracle.so`` from
``clbm_oracle.c``.  ``-ffp-contract=off`` keeps every product and sum rounded
as written, so the oracle's results are the same on x86_64 and aarch64
hosts, whatever FMA units they have.
"""
from __future__ import annotations

import os
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "clbm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")


def library_path() -> str:
    return os.path.join(OUT_DIR, "liboracle.so")


def _compile(extra):
    os.makedirs(OUT_DIR, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=OUT_DIR)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", *extra, "-o", tmp, SRC, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        os.unlink(tmp)
        return r.stderr
    os.replace(tmp, library_path())
    return None


def build(openmp: bool = True) -> str:
    """Compile the oracle; OpenMP over lattice rows when the compiler has it."""
    err = _compile(["-fopenmp"]) if openmp else "skipped"
    if err is not None:
        err2 = _compile([])
        if err2 is not None:
            raise RuntimeError("oracle build failed:\n" + err2)
    return library_path()


if __name__ == "__main__":
    print(build())
