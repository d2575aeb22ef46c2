"""Build the in-tree CUDA library libsph_b300.so for sm_103a (nvcc, no JIT cache)."""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

HERE = Path(__file__).resolve().parent
CSRC = HERE / "csrc"
INCLUDE = HERE.parent / "include"
LIB = HERE / "libsph_b300.so"
SOURCES = ["sph_kernels.cu", "sph_passes.cu", "sph_runtime.cu", "sph_server.cu", "sph_noalloc.cu", "sph_rebuild.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _stale() -> bool:
    if not LIB.exists():
        return True
    t = LIB.stat().st_mtime
    deps = list(CSRC.glob("*")) + list(INCLUDE.glob("*.h")) + [Path(__file__)]
    return any(p.stat().st_mtime > t for p in deps if p.is_file())


def build(force: bool = False, verbose: bool = False) -> Path:
    """Compile every source into one shared library next to the package."""
    if not force and not _stale():
        return LIB
    objs = []
    bdir = HERE / "_build"
    bdir.mkdir(exist_ok=True)
    flags = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
                    "--expt-relaxed-constexpr", "-I", str(INCLUDE)]
    if verbose:
        flags += ["-Xptxas", "-v"]
    for src in SOURCES:
        s = CSRC / src
        if not s.exists():
            continue
        o = bdir / (s.stem + ".o")
        subprocess.run([nvcc(), *flags, "-c", str(s), "-o", str(o)], check=True)
        objs.append(str(o))
    tmp = str(LIB) + ".tmp"
    subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
