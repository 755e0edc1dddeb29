"""Compile liblsp.so (the CUDA kernels and the C ABI of include/lsp.h) for sm_103a, in-tree.

    python -m paper_1607_02560_gb300.build

Each .cu file is compiled in parallel to an object file under _build/, then linked into
paper_1607_02560_gb300/liblsp.so. Host code is compiled without floating-point contraction so
that lattice-shift rounding decisions are plain IEEE evaluations on every host architecture.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblsp.so")
LIB_CHECKS = os.path.join(HERE, "liblsp_checks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _compile(src: str, extra: list[str], build_dir: str = BUILD) -> str:
    obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    return obj


def build(verbose: bool = False, extra: list[str] | None = None, checks: bool = False) -> str:
    """Compile and link liblsp.so; returns its path. Rebuilds only when a source is newer.

    checks=True builds liblsp_checks.so instead: the same library compiled with -DLSP_CHECKS,
    whose kernels record out-of-range indices in the error word (LSP_ERR_STATE) and keep every
    access inside its array."""
    extra = list(extra or []) + (["-DLSP_CHECKS"] if checks else [])
    lib = LIB_CHECKS if checks else LIB
    build_dir = BUILD + "_checks" if checks else BUILD
    os.makedirs(build_dir, exist_ok=True)
    srcs = sources()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "lsp.h"))
    newest = max(os.path.getmtime(p) for p in srcs + headers + [__file__])
    if os.path.exists(lib) and os.path.getmtime(lib) >= newest and (checks or not extra):
        return lib
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, build_dir), srcs))
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)
    if verbose:
        print("built", lib)
    return lib


if __name__ == "__main__":
    args = sys.argv[1:]
    build(verbose=True, extra=[a for a in args if a != "--checks"], checks="--checks" in args)
