"""Build the native library ``libhisvsim.so`` in-tree with nvcc for sm_103a.

Each translation unit compiles in parallel into ``_build/``; the shared
library is linked next to this file. Host C++ and CUDA both go through nvcc
(host code is plain C++17 with no architecture-specific flags, so the same
sources build on x86_64 and aarch64).
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
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhisvsim.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["kernels.cu", "dense.cu", "dense_pair.cu", "dense_batch.cu", "noalloc.cu", "batch.cu", "abi.cpp", "batch_abi.cpp",
           "partition.cpp", "planner.cpp", "qasm.cpp", "jit.cpp"]
# headers handed to the run-time compiler (NVRTC) by jit.cpp, embedded as
# string literals: name in the generated include file -> source header
JIT_HEADERS = (("kJitOpsCore", "ops_core.cuh"), ("kJitPrelude", "jit_prelude.cuh"))
JIT_INC = os.path.join(BUILD, "jit_sources.inc")


def _nvcc():
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhisvsim.so")


def _compile(src: str, verbose: bool) -> str:
    path = os.path.join(CSRC, src)
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    deps = [path] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".hpp", ".cuh"))]
    deps.append(os.path.join(INCLUDE, "hisvsim.h"))
    if src == "jit.cpp":
        deps.append(JIT_INC)
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(d) for d in deps):
        return obj
    cmd = [_nvcc(), "-std=c++17", "-O3", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", BUILD, "-c", path, "-o", obj]
    if src.endswith(".cu"):
        cmd[1:1] = ARCH + ["-lineinfo", "--expt-relaxed-constexpr"]
        if verbose:
            cmd += ["-Xptxas", "-v"]
    else:
        cmd += ["-x", "c++"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
    if verbose and res.stderr:
        sys.stderr.write(res.stderr)
    return obj


def _write_jit_sources():
    """The run-time compiler's headers as C++ raw string literals (rewritten
    only when their text changes, so the dependency check stays exact)."""
    text = "// generated by build.py from csrc/ops_core.cuh and csrc/jit_prelude.cuh\n"
    for name, hdr in JIT_HEADERS:
        with open(os.path.join(CSRC, hdr)) as f:
            body = f.read()
        assert ")HISVSRC" not in body
        text += f'static const char *{name} = R"HISVSRC({body})HISVSRC";\n'
    if os.path.exists(JIT_INC):
        with open(JIT_INC) as f:
            if f.read() == text:
                return
    with open(JIT_INC, "w") as f:
        f.write(text)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for f in os.listdir(BUILD):
            os.remove(os.path.join(BUILD, f))
    _write_jit_sources()
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), srcs))
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(o) for o in objs):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [_nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
