"""Builds the CUDA library libras.so for sm_103a with nvcc (in-tree).

Each translation unit is compiled in parallel, then linked with the static
CUDA runtime into paper_2007_13966_gb300/_lib/libras.so.
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
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libras.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["problem.cu", "schwarz.cu", "precond.cu", "krylov.cu", "coarse.cu", "ras125.cu",
           "noalloc.cu", "batch.cu", "tc_gemm.cu"]


def source_hash(files=None) -> str:
    """Hash of CUDA sources (all of csrc/ and the ABI header by default, or the
    named csrc/ files): identifies the build a measurement was taken on."""
    import hashlib
    h = hashlib.sha256()
    names = sorted(os.listdir(CSRC)) + ["../../include/ras.h"] if files is None else list(files)
    for fn in names:
        path = os.path.normpath(os.path.join(CSRC, fn))
        if path.endswith((".cu", ".cuh", ".h")) and os.path.isfile(path):
            h.update(os.path.basename(path).encode())
            with open(path, "rb") as f:
                h.update(f.read())
    return h.hexdigest()[:16]


# files that define the fine-level subdomain-solve kernels (k_ras_apply, k_ras_pipe):
# their own source; the shared header holds host-side declarations only
RAS_APPLY_FILES = ("schwarz.cuh", "schwarz.cu")


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def build(verbose: bool = False, jobs: int | None = None) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    obj_dir = os.path.join(OUT_DIR, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        cmd = [cc, *_flags(), "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=jobs or len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
