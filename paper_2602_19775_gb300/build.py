"""In-tree build of libssa.so for sm_103a (nvcc, no cmake).

    python -m paper_2602_19775_gb300.build

Each translation unit under csrc/ is compiled in parallel with
`-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`, then linked into
paper_2602_19775_gb300/libssa.so. The build is incremental on file modification times.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libssa.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-warn-spills"]


def _nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand) and shutil.which(cand) is None:
        raise RuntimeError("nvcc not found; set NVCC or put the CUDA toolkit on PATH")
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(PKG, "..", "include", "*.h")))


JIT_TEXT = os.path.join(OUT_DIR, "ssa_jit_text.h")
JIT_SOURCES = (("kJitTextDevice", os.path.join(CSRC, "ssa_device.cuh")),
               ("kJitTextBody", os.path.join(CSRC, "ssa_jit_body.cuh")),
               ("kJitTextApi", os.path.join(PKG, "..", "include", "ssa.h")))


def _write_jit_text():
    """The device sources compiled at run time (NVRTC), embedded in the library as string literals."""
    parts = ["// generated by build.py from csrc/ssa_device.cuh, csrc/ssa_jit_body.cuh and include/ssa.h\n#pragma once\n"]
    for name, path in JIT_SOURCES:
        text = open(path).read()
        if ")SSAJIT\"" in text:
            raise RuntimeError(f"{path} contains the raw-string delimiter")
        parts.append(f'static const char {name}[] = R"SSAJIT({text})SSAJIT";\n')
    new = "".join(parts)
    if not os.path.exists(JIT_TEXT) or open(JIT_TEXT).read() != new:
        with open(JIT_TEXT + ".tmp", "w") as f:
            f.write(new)
        os.replace(JIT_TEXT + ".tmp", JIT_TEXT)


def _compile(nvcc: str, src: str, extra: list[str]) -> str:
    obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
    newest_dep = max([os.path.getmtime(src)] + [os.path.getmtime(h) for h in _headers() + [JIT_TEXT]])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest_dep:
        return obj
    cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-I", OUT_DIR, *extra, "-c", src, "-o", obj + ".tmp"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{res.stdout}\n{res.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile every csrc/*.cu for sm_103a and link libssa.so; returns the library path."""
    nvcc = _nvcc()
    os.makedirs(OUT_DIR, exist_ok=True)
    extra = list(extra or [])
    _write_jit_text()
    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(nvcc, s, extra), srcs))
    newest = max(os.path.getmtime(o) for o in objs)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lnvrtc"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
