"""Build libfcas.so in-tree with nvcc for sm_103a (one translation unit per process, then link)."""

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfcas.so")
SOURCES = ["fcas_api.cu", "fcas_kernels.cu", "fcas_create.cu", "fcas_noalloc.cu", "fcas_pso.cu", "fcas_grad.cu",
           "fcas_diag.cu", "fcas_kernels_ff.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc():
    exe = shutil.which("nvcc")
    if exe is None and os.path.exists("/usr/local/cuda/bin/nvcc"):
        exe = "/usr/local/cuda/bin/nvcc"
    if exe is None:
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfcas.so")
    return exe


def _compile(src, verbose, defines=(), build_dir=BUILD):
    obj = os.path.join(build_dir, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), *FLAGS, *ARCH, *[f"-D{d}" for d in defines], "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(verbose=False, force=False, defines=(), out=None):
    """Compile every CUDA source and link libfcas.so next to this file (or at `out`, with extra
    preprocessor `defines` for launch-shape tuning). Returns the library path."""
    if defines or out:
        build_dir = BUILD + "_" + hashlib.sha1(" ".join(defines).encode()).hexdigest()[:8]
        target = out or LIB
        if not force and out and os.path.exists(target):
            srcs = [os.path.join(CSRC, s) for s in SOURCES]
            hdrs = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
            hdrs.append(os.path.join(HERE, "..", "include", "fcas.h"))
            if os.path.getmtime(target) >= max(os.path.getmtime(p) for p in srcs + hdrs + [__file__]):
                return target
        os.makedirs(build_dir, exist_ok=True)
        with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            objs = list(ex.map(lambda s: _compile(s, verbose, defines, build_dir), SOURCES))
        r = subprocess.run([_nvcc(), *ARCH, "-shared", "-o", target + ".tmp", *objs, "-lcudart"], capture_output=True,
                           text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(target + ".tmp", target)
        return target
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    headers.append(os.path.join(HERE, "..", "include", "fcas.h"))
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(p) for p in srcs + headers + [__file__])
        if os.path.getmtime(LIB) >= newest:
            return LIB
    os.makedirs(BUILD, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    tmp = LIB + ".tmp"
    cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
