"""Build of the CUDA library libts_gb300.so (sm_103a) in-tree, under ``_build/``.

Every translation unit is compiled by one nvcc process (in parallel) for
``-gencode arch=compute_103a,code=sm_103a`` and linked into a shared library with the shared CUDA
runtime. Device code is compiled without FMA contraction (``-fmad=false``) and host code with
``-ffp-contract=off``: the bin/subbin boundaries round exactly as written, and the exact FP64 pair
test fuses exactly the multiply-adds it writes as ``fma()``.
"""
from __future__ import annotations

import concurrent.futures
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libts_gb300.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["ts_prims.cu", "ts_index.cu", "ts_search.cu", "ts_batch.cu", "ts_server.cu",
           "ts_api.cu", "ts_noalloc.cu", "ts_peaks.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _flags():
    return [ARCH, "-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler",
            "-fPIC,-ffp-contract=off,-O2", "-I", INCLUDE, "-I", CSRC]


def _digest() -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(INCLUDE, "ts.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(_flags()).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the library if its sources changed; returns the .so path."""
    os.makedirs(OUT, exist_ok=True)
    stamp = os.path.join(OUT, "stamp.txt")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == dig:
                return LIB
    nvcc = os.path.join(cuda_home(), "bin", "nvcc")

    def compile_one(src):
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        cmd = [nvcc, *_flags(), "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, err in results:
            print(err)
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc, ARCH, "-shared", "-cudart", "shared", "-o", tmp, *[o for o, _ in results],
           "-Xlinker", f"-rpath,{os.path.join(cuda_home(), 'lib64')}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
