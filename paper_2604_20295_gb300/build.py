"""In-tree build of libetac.so for sm_103a (nvcc, one -gencode, sources compiled in parallel).

``python -m paper_2604_20295_gb300.build`` or ``build()``; the library lands in
``paper_2604_20295_gb300/_build/libetac.so`` and is rebuilt when a source or header is newer.
``build(variant=...)`` builds a variant of the same sources with extra defines into its own
folder (``_build/<variant>/libetac.so``); the binding loads it when ``ETAC_LIBRARY`` names it.
Variants: ``outline_refine`` (the exact contact decision as an out-of-line call in every
kernel, to show that inlining does not change the results); ``bounds`` (ETAC_BOUNDS: index
checks on the forward kernels' and the regressor's global writes, which latch ETAC_ERR_BOUNDS
in the device status word and skip the access instead of faulting).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libetac.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libetac")
    return cand


def sources() -> list:
    """CUDA sources and host-only C++ sources (both compiled by nvcc)."""
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps() -> list:
    return (sources() + glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h")) +
            [os.path.abspath(__file__)])


VARIANTS = {"outline_refine": ["-DETAC_OUTLINE_REFINE"], "bounds": ["-DETAC_BOUNDS"]}


def variant_lib(variant: str) -> str:
    return os.path.join(OUT_DIR, variant, "libetac.so")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), variant: str = None) -> str:
    """Compile every CUDA source for sm_103a and link libetac.so (no-op when up to date)."""
    out_dir, lib = OUT_DIR, LIB
    if variant is not None:
        extra_flags = list(extra_flags) + VARIANTS[variant]
        out_dir = os.path.join(OUT_DIR, variant)
        lib = variant_lib(variant)
    if not force and not _stale(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    flags = NVCC_FLAGS + list(extra_flags)

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.splitext(os.path.basename(src))[0] + ".o")
        cmd = [nvcc] + ARCH + flags + ["-c", src, "-o", obj]
        if verbose:
            cmd.append("-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    srcs = sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of libetac.so failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
