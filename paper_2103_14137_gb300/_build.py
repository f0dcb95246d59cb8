"""Compile libuvc.so (the C-ABI library) in-tree for sm_103a with nvcc."""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libuvc.so")
SOURCES = ["build_bvh.cu", "irradiance.cu", "batch.cu", "fluence.cu", "solid_angle.cu", "raster.cu", "features.cu", "mlp.cu", "probe.cu", "api.cu"]
HEADERS = ["uvc_internal.cuh", "traverse.cuh"]
INCLUDE = os.path.join(HERE, "..", "include")
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc():
    for p in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        c = os.path.join(p, "bin", "nvcc")
        if p and os.path.exists(c):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """libuvc.so, or with checked=True libuvc_checked.so: the same sources
    compiled with UVC_CHECKED (bounds-checked traversal indices)."""
    out = OUT if not checked else os.path.join(HERE, "libuvc_checked.so")
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(HERE, "..", "include", "uvc.h")]
    if not force and os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(d) for d in deps):
        return out
    bdir = os.path.join(HERE, "_build" if not checked else "_build_checked")
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = [nvcc, *NVCC_FLAGS, *(["-DUVC_CHECKED"] if checked else []), "-I", INCLUDE, "-c",
               os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = out + f".{os.getpid()}.tmp"
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", *objs, "-o", tmp],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out
