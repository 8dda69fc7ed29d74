"""Build the CUDA library libtdgl_gb300.so in-tree (sm_103a only).

Each translation unit is compiled in parallel with nvcc and linked into one
shared library under paper_1409_8340_gb300/_build/.  The CUDA runtime is
linked dynamically (the same libcudart.so.13 that PyTorch loads).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libtdgl_gb300.so")
SOURCES = ["tdgl_api.cu", "tdgl_resident.cu", "k_jacobi.cu", "k_poisson.cu", "k_obs.cu", "k_pattern.cu", "tdgl_noalloc.cu", "k_adjoint.cu", "tdgl_adjoint_api.cu", "k_batch.cu", "tdgl_batch_api.cu", "k_pair.cu", "k_insulating.cu", "k_sweep_tma.cu"]
HEADERS = ["tdgl_internal.cuh", "sweep_tile.cuh", "mg_tile.cuh", os.path.join("..", "..", "include", "tdgl.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def cuda_lib_dir() -> str:
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc())))
    for d in ("lib64", os.path.join("targets", "sbsa-linux", "lib"), os.path.join("targets", "x86_64-linux", "lib"), "lib"):
        if os.path.exists(os.path.join(root, d, "libcudart.so")):
            return os.path.join(root, d)
    return os.path.join(root, "lib64")


def _stale(extra_flags: list[str]) -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(CSRC, h) for h in HEADERS] + [__file__]
    if any(os.path.getmtime(d) > t for d in deps):
        return True
    stamp = os.path.join(BUILD, "flags.txt")
    return not os.path.exists(stamp) or open(stamp).read() != " ".join(extra_flags)


def build(force: bool = False, extra_flags: list[str] | None = None, verbose: bool = False) -> str:
    extra_flags = list(extra_flags or [])
    if not force and not _stale(extra_flags):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    common = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-v" if verbose else "-O3", *extra_flags]

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = common + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    libdir = cuda_lib_dir()
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "shared", f"-L{libdir}",
           "-Xlinker", f"-rpath,{libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(os.path.join(BUILD, "flags.txt"), "w") as fh:
        fh.write(" ".join(extra_flags))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
