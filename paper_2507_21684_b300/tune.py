"""Autotuner of the neighbour-search settings of a scene.

The cell edge is H + skin.  A wider skin lets the cells serve more steps (the device-side check
rebuilds them only when some particle has moved skin/2, or after `rebuild_interval` sweeps) but
every sweep then tests more candidates.  The best trade depends on the scene's particle speed,
time step and size, so it is measured: each candidate runs on the device through the public API
(the same graph-captured steps a caller gets) and the fastest mean step time wins.  The physics
does not depend on the choice: every candidate finds the same neighbours (|r| < H) each step.
"""
from __future__ import annotations

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
              chunk: int = 1) -> dict:
    """Time each skin (a fraction of H) on `spec` and return the best parameters with the table."""
    table = []
    for f in skins:
        r = time_steps(with_skin(spec, f, interval), steps=steps, warmup=warmup, chunk=chunk)
        table.append(dict(skin_over_H=float(f), **r))
    best = min(table, key=lambda r: r["ms_per_step"])
    return {"params": with_skin(spec, best["skin_over_H"], interval)["params"], "best": best, "table": table}
