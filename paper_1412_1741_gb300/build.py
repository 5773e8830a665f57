"""Build libparem.so (the CUDA path) from csrc/ with nvcc for sm_103a.

Each translation unit compiles in its own nvcc process, in parallel, then one link step
makes the shared library.  The result lands in paper_1412_1741_gb300/_build/ (git-ignored)
and is rebuilt when a source is newer than it.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libparem.so")
SOURCES = ["parem_api.cu", "parem_prep.cpp", "parem_k_byte.cu", "parem_k_class.cu", "parem_k_global.cu",
           "parem_noalloc.cu", "parem_k_batch.cu", "parem_batch.cu", "parem_server.cpp", "parem_k_win.cu",
           "parem_regex.cpp", "parem_k_pair.cu", "parem_pair.cpp"]
HEADERS = ["parem_internal.h", "parem_launch.h", "parem_scan.cuh", "parem_batch_impl.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags():
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
            f"-I{os.path.join(ROOT, 'include')}", "--expt-relaxed-constexpr"] + ARCH


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, verbose=False):
    obj = os.path.join(BUILD, src + ".o")
    deps = [os.path.join(CSRC, src)] + [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "parem.h")]
    if not _stale(obj, deps):
        return obj
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj + ".tmp"] + _flags()
    if src.endswith(".cpp"):
        cmd = [nvcc(), "-x", "cu", "-c", os.path.join(CSRC, src), "-o", obj + ".tmp"] + _flags()
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for f in os.listdir(BUILD):
            os.remove(os.path.join(BUILD, f))
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    if _stale(LIB, objs):
        cmd = [nvcc(), "-shared", "-o", LIB + ".tmp"] + objs + ARCH + ["-cudart", "shared", "-Xlinker", "-rpath=/usr/local/cuda/lib64"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
