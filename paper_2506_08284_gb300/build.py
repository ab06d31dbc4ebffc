"""Compile the sm_103a CUDA sources of the library into ``_build/libsphc.so``.

nvcc -gencode arch=compute_103a,code=sm_103a, one object per translation unit (compiled in
parallel), linked as a plain shared library exporting the C ABI of ``include/sphc.h``.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["sparse.cu", "setup.cu", "layout.cu", "solve.cu", "block.cu", "capi.cu", "noalloc.cu", "mlp.cu", "cond.cu"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden", "--expt-relaxed-constexpr"]


def _digest() -> str:
    h = hashlib.sha1()
    for name in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(ROOT, "include", "sphc.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(FLAGS).encode())
    return h.hexdigest()[:12]


def library_path() -> str:
    return os.path.join(BUILD, f"libsphc_{_digest()}.so")


def build(force: bool = False, verbose: bool = False) -> str:
    so = library_path()
    if os.path.exists(so) and not force:
        return so
    os.makedirs(BUILD, exist_ok=True)
    tag = os.path.basename(so)[len("libsphc_"):-3]
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD, f"{src[:-3]}_{tag}.o")
        cmd = [NVCC, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = so + f".tmp{os.getpid()}"
    r = subprocess.run([NVCC, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp, *objs,
                        "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, so)
    for o in objs:
        os.remove(o)
    for name in os.listdir(BUILD):                       # drop libraries of older sources
        if name.startswith("libsphc_") and name.endswith(".so") and name != os.path.basename(so):
            try:
                os.remove(os.path.join(BUILD, name))
            except OSError:
                pass
    return so


if __name__ == "__main__":
    print(build(force=True, verbose=True))
