"""Builds the CUDA library liblrdmc.so in place (nvcc, sm_103a only), and
its bounds-checked variant liblrdmc_bounds.so (-DLRDMC_BOUNDS: walker-level
indices checked on the device, LRDMC_ERR_BOUNDS on a violation)."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "liblrdmc.so")
LIB_BOUNDS = os.path.join(HERE, "liblrdmc_bounds.so")
SOURCES = ["lrdmc_kernels.cu", "lrdmc_api.cu", "lrdmc_neural.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "lrdmc.h"))
    return files


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    """Compile liblrdmc.so (liblrdmc_bounds.so with bounds=True) unless it is
    newer than every source. Extra nvcc flags (tuning macros such as
    -DLRDMC_DF_OUTLINE) come from the environment variable LRDMC_NVCC_FLAGS."""
    lib = LIB_BOUNDS if bounds else LIB
    if not force and os.path.exists(lib):
        newest = max(os.path.getmtime(f) for f in _inputs())
        if os.path.getmtime(lib) >= newest:
            return lib
    build_dir = os.path.join(HERE, "_build_bounds" if bounds else "_build")
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if verbose else []
    extra += os.environ.get("LRDMC_NVCC_FLAGS", "").split()
    if bounds:
        extra.append("-DLRDMC_BOUNDS")

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static" if False else "-cudart=static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> list[str]:
    """Both libraries, compiled concurrently."""
    with ThreadPoolExecutor(max_workers=2) as ex:
        return list(ex.map(lambda b: build(force=force, bounds=b), (False, True)))


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, bounds="--bounds" in sys.argv))
