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
# Tile-shape variants of the library (targets per tile, threads per target, threads per CTA, staged
# capacity, hit-list length, line cutting, for 2D and 3D), timed against each other by
# tune.tune_tiles; "default" is libsph_b300.so.
VARIANTS = {
    "default": {},
    "lanes8": {"SPH_TILE2_TP": 32, "SPH_TILE2_LANES": 8, "SPH_TILE2_LIST": 16,
               "SPH_TILE3_TP": 16, "SPH_TILE3_LANES": 16, "SPH_TILE3_LIST": 12},
    "lanes2": {"SPH_TILE2_TP": 128, "SPH_TILE2_LANES": 2, "SPH_TILE2_LIST": 40},
    "small": {"SPH_TILE2_TP": 32, "SPH_TILE2_LANES": 4, "SPH_TILE2_LIST": 24, "SPH_TILE2_THREADS": 128,
              "SPH_TILE2_CAP": 512},
    # the same 2D tiles with the cooperative rebuild on one CTA per SM (a cheaper launch on the
    # steps that rebuild nothing, a slower rebuild when one is due)
    "small1": {"SPH_TILE2_TP": 32, "SPH_TILE2_LANES": 4, "SPH_TILE2_LIST": 24, "SPH_TILE2_THREADS": 128,
               "SPH_TILE2_CAP": 512, "SPH_RB_CTAS_PER_SM": 1},
    "small3": {"SPH_TILE3_TP": 16, "SPH_TILE3_LANES": 8, "SPH_TILE3_LIST": 18, "SPH_TILE3_THREADS": 128,
               "SPH_TILE3_CAP": 768},
    # how lines are cut into tiles: whole cells in 2D, whole cells in 3D (the defaults swapped)
    "cells2": {"SPH_TILE2_CUT": 0},
    "cells3": {"SPH_TILE3_CUT": 0},
    # the 3D sweep on the staged traversal instead of the warp-per-tile one (with its whole-cell cut)
    "staged3": {"SPH_W3": 0, "SPH_TILE3_CUT": 0},
    # the warp-per-tile 3D sweep with 8 candidates (4 paired loads) per step of the test loop
    # (default 16)
    "w3u8": {"SPH_W_UNROLL": 8},
    # the 3D sweep's evaluation one hit per iteration (default two)
    "w3d1": {"SPH_W_DRAIN2": 0},
    # 4 x sub-bins per cell in the 3D sweep's keys (default 8)
    "w3b4": {"SPH_W_XSHIFT": 2},
    # the cooperative rebuild on one CTA per SM (a cheaper launch on the steps that rebuild nothing)
    "rb1": {"SPH_RB_CTAS_PER_SM": 1},
    # the 3D sweep's earlier schedule: CTAs of 4 warps at 5 per SM, every warp claiming its own tiles
    # from the launch's counter, 32-entry hit rings (default: one CTA of 24 warps per SM taking
    # chunks of 8 tiles, 16-entry rings)
    "w3w4": {"SPH_W_WARPS": 4, "SPH_W_MINB": 5, "SPH_W_CHUNK": 0, "SPH_W_LIST": 32},
    # chunks of 12 tiles
    "w3c12": {"SPH_W_CHUNK": 12},
    # captured 3D steps with a skin rebuild in one cooperative launch instead of a conditional
    # graph node (the same kernels; ncu can profile these graphs)
    "coop3": {"SPH_COOP3": 1},
}


def variant_macros(variant: str) -> dict:
    """Macros of a variant; "a+b" combines two variants that set different dimensions' shapes
    (the autotuner's 3D choice with its 2D one)."""
    parts = [p for p in variant.split("+") if p and p != "default"]
    out: dict = {}
    for p in parts:
        if p not in VARIANTS:
            raise ValueError(f"unknown library variant {p!r}")
        for k, v in VARIANTS[p].items():
            if k in out and out[k] != v:
                raise ValueError(f"variants in {variant!r} disagree on {k}")
            out[k] = v
    return out


def canonical(variant: str) -> str:
    """One name per combination: the non-default parts in VARIANTS order, joined by "+"."""
    parts = {p for p in variant.split("+") if p and p != "default"}
    variant_macros(variant)  # validates
    names = [v for v in VARIANTS if v in parts]
    return "+".join(names) if names else "default"


def lib_path(variant: str = "default") -> Path:
    variant = canonical(variant)
    return LIB if variant == "default" else HERE / f"libsph_b300_{variant.replace('+', '_')}.so"


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _stale(lib: Path = LIB) -> bool:
    if not lib.exists():
        return True
    t = lib.stat().st_mtime
    deps = list(CSRC.glob("*")) + list(INCLUDE.glob("*.h")) + [Path(__file__)]
    return any(p.stat().st_mtime > t for p in deps if p.is_file())


def build(force: bool = False, verbose: bool = False, variant: str = "default") -> Path:
    """Compile every source into one shared library next to the package (one tile-shape variant)."""
    variant = canonical(variant)
    lib = lib_path(variant)
    if not force and not _stale(lib):
        return lib
    objs = []
    bdir = HERE / "_build" / variant.replace("+", "_")
    bdir.mkdir(parents=True, exist_ok=True)
    flags = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
                    "--expt-relaxed-constexpr", "-I", str(INCLUDE)]
    flags += [f"-D{k}={v}" for k, v in variant_macros(variant).items()]
    if verbose:
        flags += ["-Xptxas", "-v"]
    jobs = []
    for src in SOURCES:
        s = CSRC / src
        if not s.exists():
            continue
        o = bdir / (s.stem + ".o")
        jobs.append([nvcc(), *flags, "-c", str(s), "-o", str(o)])
        objs.append(str(o))
    # one nvcc process per source, in parallel
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for f in [ex.submit(subprocess.run, j, check=True) for j in jobs]:
            f.result()
    tmp = str(lib) + ".tmp"
    subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], check=True)
    os.replace(tmp, lib)
    return lib


def build_all(force: bool = False) -> list:
    """Every tile-shape variant (the default first; the variants in parallel)."""
    first = build(force=force)
    from concurrent.futures import ThreadPoolExecutor
    rest = [v for v in VARIANTS if v != "default"]
    with ThreadPoolExecutor(max_workers=max(1, len(rest))) as ex:
        libs = [f.result() for f in [ex.submit(build, force, False, v) for v in rest]]
    return [first] + libs


if __name__ == "__main__":
    if "--all" in sys.argv:
        for p in build_all(force="--force" in sys.argv):
            print(p)
    else:
        print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
