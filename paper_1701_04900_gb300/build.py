"""Build the CUDA C-ABI library ``libasyflexa.so`` in-tree for sm_103a with nvcc.

Each translation unit compiles in parallel; the result is linked with the static CUDA
runtime so the library only needs the CUDA driver at run time.  Usage:

    python -m paper_1701_04900_gb300.build          # build if sources changed
    python -m paper_1701_04900_gb300.build --force  # always rebuild
"""

from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libasyflexa.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
UNITS = ["api.cu", "inst_f64.cu", "inst_f32.cu", "inst_bf16.cu", "inst_fp8.cu", "noalloc.cu", "quantize.cu",
         "batch.cu", "multi.cu", "selftest.cu", "adjoint.cu"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libasyflexa")


def _flags(extra=()):
    return [ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", INCLUDE, "-I", CSRC,
            "--expt-relaxed-constexpr", *extra]


def _digest() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            p = os.path.join(d, name)
            if os.path.isfile(p):
                h.update(name.encode())
                with open(p, "rb") as f:
                    h.update(f.read())
    h.update(" ".join(_flags()).encode())
    return h.hexdigest()


def build_library(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    """Compile and link ``libasyflexa.so``; returns its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    stamp = os.path.join(OUT_DIR, "build.sha256")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == dig:
                return LIB
    nvcc = _nvcc()
    objs = []
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []

    def compile_one(unit):
        src = os.path.join(CSRC, unit)
        obj = os.path.join(OUT_DIR, unit.replace(".cu", ".o"))
        cmd = [nvcc, *_flags(extra), "-c", src, "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {unit}:\n{res.stderr}\n{res.stdout}")
        return obj, res.stderr

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        for obj, log in ex.map(compile_one, UNITS):
            objs.append(obj)
            if verbose and log:
                sys.stderr.write(log)
    tmp = LIB + ".tmp"
    cmd = [nvcc, ARCH, "-shared", "-Xcompiler", "-fPIC", "-cudart", "static", "-o", tmp, *objs]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stderr}\n{res.stdout}")
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    force = "--force" in sys.argv
    path = build_library(force=force, verbose="-v" in sys.argv, ptxas_verbose="--ptxas" in sys.argv)
    print(path)
