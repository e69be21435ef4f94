"""Build libcroft.so (the C-ABI library) in-tree with nvcc for sm_103a.

Translation units compile in parallel; the pass-kernel instantiations are split
into four size groups (``croft_kernels.cu`` compiled with ``-DCROFT_GROUP=g``),
the fused convolution pass into five (``croft_conv.cu``, ``-DCROFT_CONV_GROUP=g``).
Objects go to ``paper_2002_04896_gb300/_build/`` and are rebuilt only when a
source or header is newer than the object.
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
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libcroft.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", CSRC, "-I", os.path.join(ROOT, "include")]
N_GROUPS = 4


def nvcc_path() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libcroft")


def _units():
    units = []
    for g in range(N_GROUPS):
        units.append((os.path.join(CSRC, "croft_kernels.cu"), os.path.join(BUILD, f"croft_kernels_g{g}.o"),
                      [f"-DCROFT_GROUP={g}"]))
    for g in range(5):
        units.append((os.path.join(CSRC, "croft_conv.cu"), os.path.join(BUILD, f"croft_conv_g{g}.o"),
                      [f"-DCROFT_CONV_GROUP={g}"]))
    for g in range(4):
        units.append((os.path.join(CSRC, "croft_tc.cu"), os.path.join(BUILD, f"croft_tc_g{g}.o"),
                      [f"-DCROFT_TC_GROUP={g}"]))
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        if os.path.basename(src) in ("croft_kernels.cu", "croft_conv.cu"):
            continue
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        units.append((src, obj, []))
    return units


def _deps_mtime() -> float:
    files = glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def _compile(unit, verbose: bool):
    src, obj, extra = unit
    cmd = [nvcc_path()] + ARCH + NVCC_FLAGS + extra + ["-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)} {extra}:\n{r.stderr}")
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if needed) and link libcroft.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    newest = _deps_mtime()
    units = _units()
    todo = [u for u in units if force or not os.path.exists(u[1]) or os.path.getmtime(u[1]) < newest]
    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(len(todo), os.cpu_count() or 4)) as ex:
            for obj, log in ex.map(lambda u: _compile(u, verbose), todo):
                if verbose and log:
                    sys.stderr.write(log)
    objs = [u[1] for u in units]
    if force or todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + ".tmp"
        cmd = [nvcc_path()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-ldl", "-lrt", "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


def ensure_built() -> str:
    return build(force=False)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
