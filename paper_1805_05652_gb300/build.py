"""Build libfmap.so (CUDA C++ for sm_103a) in-tree: ``_lib/libfmap.so``.

Each translation unit is compiled in parallel with nvcc, then linked as a
shared library exporting the C ABI of ``include/fmap.h``.
"""

from __future__ import annotations

import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

_HERE = os.path.dirname(os.path.abspath(__file__))
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-Xptxas", "-O3"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def lib_path() -> str:
    return os.path.join(_HERE, "_lib", "libfmap.so")


def sources():
    return sorted(glob.glob(os.path.join(_HERE, "csrc", "*.cu")))


def _deps():
    files = sources() + glob.glob(os.path.join(_HERE, "csrc", "*.h")) + \
        glob.glob(os.path.join(_HERE, "csrc", "*.cuh")) + \
        glob.glob(os.path.join(_HERE, "..", "include", "*.h"))
    return files


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    out = lib_path()
    if not force and os.path.exists(out):
        newest = max(os.path.getmtime(f) for f in _deps())
        if os.path.getmtime(out) >= newest:
            return out
    obj_dir = os.path.join(_HERE, "_lib", "obj")
    os.makedirs(obj_dir, exist_ok=True)
    nv = nvcc()

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
        cmd = [nv, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr.strip():
            print(r.stderr, flush=True)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nv, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lcuda"]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True, verbose=True))
