"""Builds liblassogs.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a -lineinfo -O3`` and linked into
``paper_1505_03410_gb300/_build/liblassogs.so`` against the shared CUDA
runtime.  No GPU is needed to build.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblassogs.so")
SOURCES = ["api.cu", "path.cu", "path_k_single_f32.cu", "path_k_single_f64.cu", "path_k_enet.cu", "path_k_enet_f64.cu",
           "path_k_batch.cu", "path_k_batch_enet.cu", "sparse_path.cu",
           "static_scratch.cu", "gemm_tc.cu", "lista.cu", "xtr.cu", "tune.cu"]
HEADERS = ["dfloat.cuh", "device_util.cuh", "cd_common.cuh", "gram_chain.cuh", "path_kernel.cuh", "internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblassogs")
    return cand


def _cuda_lib_dir(nvcc):
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    for d in ("lib64", "lib", os.path.join("targets", "sbsa-linux", "lib"),
              os.path.join("targets", "x86_64-linux", "lib")):
        p = os.path.join(root, d)
        if os.path.exists(os.path.join(p, "libcudart.so")):
            return p
    return os.path.join(root, "lib64")


def _stale(outputs, inputs):
    if not all(os.path.exists(o) for o in outputs):
        return True
    t_out = min(os.path.getmtime(o) for o in outputs)
    return any(os.path.getmtime(i) > t_out for i in inputs)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if needed) and return the path of liblassogs.so."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(HERE, "..", "include", h)
                                                        for h in ("lassogs.h", "lista.h")]
    objs, procs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale([o], [s] + hdrs):
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                   "-I", os.path.join(HERE, "..", "include"), "-c", s, "-o", o + ".tmp"]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), o, cmd))
    for p, o, cmd in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed ({' '.join(cmd)}):\n{out.decode(errors='replace')}")
        os.replace(o + ".tmp", o)
    if force or _stale([LIB], objs):
        libdir = _cuda_lib_dir(nvcc)
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
               "-Xlinker", f"-rpath,{libdir}", "-L", libdir]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed ({' '.join(cmd)}):\n{r.stdout}{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
