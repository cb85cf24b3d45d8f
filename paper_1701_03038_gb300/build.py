"""Build libfstgpu.so (sm_103a) in-tree with nvcc.

The library does not link libtorch: it is a plain C-ABI shared object with
the CUDA runtime linked statically, so it loads the same way under any
PyTorch version.  Translation units compile in parallel.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libfstgpu.so"
LIB_PATH = os.path.join(OUT_DIR, LIB_NAME)

SOURCES = ["sort_scan.cu", "store.cu", "kernels.cu", "capi.cu", "plan.cu", "noalloc.cu", "fd64.cu", "slice.cu",
           "train.cu", "lattice.cu", "prefix.cu", "block.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
              "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfstgpu.so")


def _newest_input() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    paths.append(os.path.join(INCLUDE, "fstgpu.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def up_to_date() -> bool:
    return os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= _newest_input()


def build(force: bool = False, verbose: bool = False, extra_flags=(), out_path: str | None = None) -> str:
    """Compile every translation unit and link libfstgpu.so; returns its path.
    ``extra_flags`` (e.g. -D tuning macros) and ``out_path`` build a variant
    elsewhere without touching the in-tree library."""
    lib_path = out_path or LIB_PATH
    if not force and not extra_flags and out_path is None and up_to_date():
        return LIB_PATH
    obj_dir = OUT_DIR if out_path is None else os.path.dirname(os.path.abspath(out_path))
    os.makedirs(obj_dir, exist_ok=True)
    cc = nvcc()
    objs = []

    def compile_one(src):
        tag = "" if out_path is None else "_" + os.path.splitext(os.path.basename(out_path))[0]
        obj = os.path.join(obj_dir, os.path.splitext(src)[0] + tag + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-ldl", "-lpthread", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))


def build_debug(out_path: str | None = None) -> str:
    """The bounds-checked variant (-DFST_DEBUG): the frontier kernels check
    their computed indices against their buffers and record violations
    (fst_debug_checks).  Built beside the in-tree library, or at out_path;
    load it with FSTGPU_LIB."""
    return build(extra_flags=["-DFST_DEBUG"], out_path=out_path or os.path.join(OUT_DIR, "libfstgpu_debug.so"))
