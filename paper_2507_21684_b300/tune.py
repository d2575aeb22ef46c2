"""Autotuner of the neighbour-search settings of a scene.

Re-sort interval: the cell edge is H + skin.  A wider skin lets the cells serve more steps (the
device-side check rebuilds them only when some particle has moved skin/2, or after
`rebuild_interval` sweeps) but every sweep then tests more candidates.  Threads per particle and
cell-block size: the library is built in tile-shape variants (targets per tile, threads per
target, build.VARIANTS); `tune_tiles` times each variant in its own process (a library is loaded
once per process) and returns the fastest, which `paper_2507_21684_b300.select_variant` then
loads.  The best choices depend on the scene's particle speed, time step and size, so they are
measured: each candidate runs on the device through the public API (the same graph-captured steps
a caller gets) and the fastest mean step time wins.  The physics does not depend on the choice:
every candidate finds the same neighbours (|r| < H) each step.
"""
from __future__ import annotations

import json
import os
import subprocess
import sys
import tempfile

import numpy as np

DEFAULT_SKINS = (0.0, 0.02, 0.05, 0.1, 0.2, 0.3)


def with_skin(spec: dict, skin_over_H: float, interval: int = 1 << 20) -> dict:
    """The scene with a Verlet skin of skin_over_H * H (0: rebuild every step)."""
    p = dict(spec["params"])
    p["skin"] = float(np.float32(skin_over_H * p["H"]))
    p["rebuild_interval"] = int(interval if skin_over_H > 0 else 1)
    return dict(spec, params=p)


def time_steps(spec: dict, steps: int = 64, warmup: int = 16, chunk: int = 1) -> dict:
    """Mean device time per step (CUDA events on the scene's stream) of `steps` steps after
    `warmup` untimed ones, issued `chunk` steps per call."""
    import torch

    import paper_2507_21684_b300 as sph
    stream = torch.cuda.Stream()
    with sph.scene_from(spec, stream=stream.cuda_stream) as sc:
        sc.step(warmup)
        s0 = sc.stats()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        done = 0
        while done < steps:
            c = min(chunk, steps - done)
            sc.step(c)
            done += c
        e1.record(stream)
        torch.cuda.synchronize()
        s1 = sc.stats()
    return {"ms_per_step": e0.elapsed_time(e1) / steps, "rebuilds": s1["rebuilds"] - s0["rebuilds"],
            "launches": s1["launches"] - s0["launches"]}


def tune_skin(spec: dict, skins=DEFAULT_SKINS, interval: int = 1 << 20, steps: int = 64, warmup: int = 16,
              chunk: int = 1, tie: float = 0.02) -> dict:
    """Time each skin (a fraction of H) on `spec` and return the best parameters with the table.
    Skins within `tie` (relative) of the fastest count as equal, and the smallest of them wins:
    its cells are the smallest, so each sweep stages and tests the fewest candidates, which also
    costs least when the state comes from DRAM rather than L2 (the timing runs steps back to back,
    with the state resident)."""
    table = []
    for f in skins:
        r = time_steps(with_skin(spec, f, interval), steps=steps, warmup=warmup, chunk=chunk)
        table.append(dict(skin_over_H=float(f), **r))
    fastest = min(r["ms_per_step"] for r in table)
    best = min((r for r in table if r["ms_per_step"] <= (1.0 + tie) * fastest), key=lambda r: r["skin_over_H"])
    return {"params": with_skin(spec, best["skin_over_H"], interval)["params"], "best": best, "table": table}


def save_spec(spec: dict, path: str) -> None:
    """A scene dict (sph_inputs) as an .npz file (arrays, and the rest as JSON)."""
    arrays = {k: v for k, v in spec.items() if isinstance(v, np.ndarray)}
    rest = {k: v for k, v in spec.items() if not isinstance(v, np.ndarray)}
    np.savez(path, __json__=np.array(json.dumps(rest)), **arrays)


def load_spec(path: str) -> dict:
    z = np.load(path)
    spec = json.loads(str(z["__json__"]))
    for k in z.files:
        if k != "__json__":
            spec[k] = z[k]
    return spec


def time_variant(variant: str, spec: dict, steps: int = 100, warmup: int = 50, device: int = 0) -> dict:
    """time_steps of `spec` with one tile-shape variant of the library, in a child process."""
    from . import build
    build.build(variant=variant)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "spec.npz")
        save_spec(spec, path)
        env = dict(os.environ, SPH_B300_VARIANT=variant)
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        out = subprocess.run([sys.executable, "-m", "paper_2507_21684_b300.tune", "--spec", path, "--steps", str(steps),
                              "--warmup", str(warmup), "--device", str(device)],
                             cwd=root, env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def shape_variants(dim: int) -> list:
    """The library variants whose tile shape differs for scenes of dimension `dim` (the default
    first): a variant that only sets the other dimension's shape runs the default one."""
    from . import build
    return [v for v, d in build.VARIANTS.items()
            if v == "default" or any(k.startswith(f"SPH_TILE{dim}_") or k == f"SPH_W{dim}" or
                                     (dim == 3 and k.startswith("SPH_W_")) for k in d)]


def tune_tiles(spec: dict, variants=None, steps: int = 100, warmup: int = 50, device: int = 0) -> dict:
    """Time every tile-shape variant for the scene's dimension on `spec`; the fastest one's name
    and the table."""
    variants = shape_variants(int(spec["params"]["dim"])) if variants is None else list(variants)
    table = []
    for v in variants:
        r = time_variant(v, spec, steps, warmup, device)
        r["variant"] = v
        table.append(r)
    best = min(table, key=lambda r: r["ms_per_step"])
    return {"variant": best["variant"], "best": best, "table": table}


def _main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="time one scene with the library variant of SPH_B300_VARIANT")
    ap.add_argument("--spec", required=True)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--device", type=int, default=0)
    a = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(a.device)
    import paper_2507_21684_b300 as sph
    sph.use_torch_allocator()
    r = time_steps(load_spec(a.spec), steps=a.steps, warmup=a.warmup)
    r["variant"] = os.environ.get("SPH_B300_VARIANT", "default")
    print(json.dumps(r))


if __name__ == "__main__":
    _main()
