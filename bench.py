"""Benchmark of the B300 WCSPH library (one JSON line on rank 0).

Headline: forward pair interactions per second on the 3D periodic Taylor-Green vortex at 128^3 =
2,097,152 particles (Wendland C2, support 2.43 dx), one bench step = one full SPH step (cell keys,
radix sort, cell ranges, permute, fused sweep with kick-drift) replayed as a CUDA graph; the
state (235 MB) exceeds L2, so no flush is needed between steps.  Beside it on the same workload:
the end-to-end call with host buffers, the FP64 oracle on the host cores (the CPU baseline) and
the FP32-vs-FP64 error of every step of a 20-step rollout.  Extra sections measure the 2D dam
break (and its renormalised, shifted, mDBC and summation variants), the adjoint rollout (128^2,
200 steps, checkpoints every 20), shifting by optimisation and the served mixed-size stream.
``--impl reference`` times the FP64 CPU oracle on the headline workload.  Multi-GPU runs are
independent replicas (the method has no data exchange between scenes): value = all ranks' pairs /
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pair interactions/s (fwd, adjoint); batched-vs-plain particle-steps/s, p99 latency"
UNIT = "pair interactions/s"
# Algorithmic FP32 flops of one in-radius ordered pair in the fused sweep (FMA = 2): the pair
# terms of the method as written, unfolded (minimum image, r^2, |r| and q, kernel gradient, Tait
# pressure of the neighbour, volume, continuity, delta diffusion, pressure, viscosity, the
# accumulations), about 80 in 2D and 3D; rejected candidates are not counted.
FLOPS_PER_PAIR = {2: 80, 3: 80}
# FP32 peak from unit counts and the maximum SM clock: 148 SMs x 128 FP32 lanes x 2 x 2.032 GHz.
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12


# Kernel sources whose change invalidates a stored ncu traffic figure.
KERNEL_SOURCES = ("sph_device.cuh", "sph_tiles.cuh", "sph_tilebuild.cuh", "sph_warptiles.cuh", "sph_passes.cuh",
                  "sph_passes.cu", "sph_kernels.cuh", "sph_kernels.cu")


def kernel_fingerprint() -> str:
    """sha256 of the kernel sources with comments and blank lines removed (a comment edit leaves
    the compiled kernels, and so a stored capture, as they were)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2507_21684_b300", "csrc", f)) as fh:
            txt = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in txt.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()[:16]


def _shape_macros(variant: str) -> dict:
    """The macros of a library variant that shape the neighbour-pass kernels (tile shape and the
    3D warp traversal); variants that differ only elsewhere (the rebuild launch) run the same
    sweep kernels."""
    from paper_2507_21684_b300 import build as sbuild
    try:
        m = sbuild.variant_macros(variant)
    except ValueError:
        return {"?": variant}
    return {k: v for k, v in m.items() if k.startswith("SPH_TILE") or k.startswith("SPH_W")}


def stored_traffic(prefix: str, variant: str = "default"):
    """DRAM bytes per launch from the committed ncu summary profiles/<prefix>*.md taken with the
    same kernel sources and a library variant of the same tile shape (the summary records both),
    with the summary's name; (None, None) when there is none."""
    import glob
    import re
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", prefix + "*.md"))):
        with open(path) as fh:
            txt = fh.read()
        fp = re.search(r"fingerprint[^`]*`([0-9a-f]+)`", txt)
        tb = re.search(r"DRAM bytes per launch \(read \+ write\): (\d+)", txt)
        lv = re.search(r"Library variant[^`]*`(\w+)`", txt)
        if (fp and tb and fp.group(1) == kernel_fingerprint()
                and _shape_macros(lv.group(1) if lv else "default") == _shape_macros(variant)):
            return int(tb.group(1)), "profiles/" + os.path.basename(path)
    return None, None


def stored_l2_bytes(source):
    """L2 bytes per launch (32 B sectors, `lts__t_sectors.sum`) of the summary stored_traffic found."""
    import re
    if not source:
        return None
    with open(os.path.join(ROOT, source)) as fh:
        m = re.search(r"`lts__t_sectors\.sum`\) \| ([0-9.]+)", fh.read())
    return float(m.group(1)) * 32.0 if m else None


def hbm_view(alg_bytes: float, dram_bytes, ms: float, peak_gbs, l2_bytes=None):
    """A kernel's algorithmic, measured DRAM and measured L2 bandwidth (bytes of one ncu launch
    over the kernel's mean time) against the measured HBM peak."""
    if not ms or ms <= 0:
        return None
    alg = alg_bytes / (ms * 1e-3) / 1e9
    dram = dram_bytes / (ms * 1e-3) / 1e9 if dram_bytes else None
    l2 = l2_bytes / (ms * 1e-3) / 1e9 if l2_bytes else None
    return {"algorithmic_gbs": alg, "dram_gbs": dram, "l2_gbs": l2, "peak_gbs": peak_gbs,
            "algorithmic_frac": alg / peak_gbs if peak_gbs else None,
            "dram_frac": dram / peak_gbs if (peak_gbs and dram) else None,
            "l2_over_hbm_peak": l2 / peak_gbs if (peak_gbs and l2) else None}


def replica_reduce(t_local: float, units_local: float, device: str = "cpu"):
    """Whole-job figures of replicas: the slowest rank's time and the units of all ranks
    (identity for a single process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t_local, units_local
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.barrier()
    return float(t.item()), float(u.item())


def replica_choice(value):
    """Rank 0's value on every rank (one configuration for all replicas)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    box = [value]
    dist.broadcast_object_list(box, src=0)
    return box[0]


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int = 0):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait(timeout=5)
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _l2_flusher(torch, stream):
    buf = torch.empty(320 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def flush():
        with torch.cuda.stream(stream):
            buf.fill_(1.0)
    return flush


def run_forward(sph, torch, spec, steps, warmup, flush_l2: bool, stream, prof_steps: int = 50, eager: bool = False):
    """Time `steps` single SPH steps (one graph launch each, CUDA events on the scene's stream),
    then profile `prof_steps` more with event nodes around each kernel class (outside the timed
    region) for the per-kernel breakdown."""
    with torch.cuda.stream(stream):
        sc = sph.scene_from(spec, stream=stream.cuda_stream)
    if eager:
        sc.set_execution(False)
    sc.step(warmup)
    flush = _l2_flusher(torch, stream) if flush_l2 else None
    torch.cuda.synchronize()
    st0 = sc.stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        if flush:
            flush()
        ev[k][0].record(stream)
        sc.step(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    st1 = sc.stats()
    ms = [a.elapsed_time(b) for a, b in ev]
    pairs_per_step, _ = sc.counters()
    sc.profile(True)
    sc.step(1)  # capture the profiled one-step graph
    sc.timing(sph.TIMING_SWEEP)
    sc.timing(sph.TIMING_REBUILD)
    sc.timing(sph.TIMING_WALLS)
    sc.timing(sph.TIMING_GRADIENT)
    sc.timing(sph.TIMING_SHIFT)
    sc.timing(sph.TIMING_DENSITY)
    for k in range(prof_steps):
        if flush:
            flush()
        sc.step(1)
    torch.cuda.synchronize()
    sweep_ms, sweep_n = sc.timing(sph.TIMING_SWEEP)
    reb_ms, reb_n = sc.timing(sph.TIMING_REBUILD)
    wall_ms, wall_n = sc.timing(sph.TIMING_WALLS)
    grad_ms, grad_n = sc.timing(sph.TIMING_GRADIENT)
    shift_ms, shift_n = sc.timing(sph.TIMING_SHIFT)
    dens_ms, dens_n = sc.timing(sph.TIMING_DENSITY)
    sc.close()
    return dict(ms=ms, pairs_per_step=pairs_per_step, launches=st1["launches"] - st0["launches"],
                rebuilds=st1["rebuilds"] - st0["rebuilds"], sweep_ms=sweep_ms / max(sweep_n, 1), sweep_n=sweep_n,
                rebuild_ms=reb_ms / max(reb_n, 1), walls_ms=wall_ms / max(wall_n, 1),
                gradient_ms=grad_ms / max(grad_n, 1), shift_ms=shift_ms / max(shift_n, 1),
                density_ms=dens_ms / max(dens_n, 1))


def run_e2e(sph, torch, spec, n_steps, reps):
    """Public-API call with host buffers: pinned host arrays in, n_steps, host arrays out."""
    stream = torch.cuda.Stream()
    pin = {k: torch.from_numpy(np.ascontiguousarray(spec[k])).pin_memory() for k in ("x", "v", "rho", "mass")}
    n, d = spec["x"].shape
    out = [torch.empty((n, d), dtype=torch.float32).pin_memory(), torch.empty((n, d), dtype=torch.float32).pin_memory(),
           torch.empty((n,), dtype=torch.float32).pin_memory()]
    lib = sph.lib()
    import ctypes as C
    times = []
    pairs = 0
    for r in range(reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p = sph.Params.from_dict(spec["params"])
        h = C.c_void_p()
        sph._check(lib.sph_init(C.byref(p), spec["n_fluid"], spec["n_wall"], pin["x"].data_ptr(), pin["v"].data_ptr(),
                                pin["rho"].data_ptr(), pin["mass"].data_ptr(), 0, C.c_void_p(stream.cuda_stream),
                                C.byref(h)))
        sph._check(lib.sph_step(h, n_steps))
        sph._check(lib.sph_get_state(h, out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), 0))
        t1 = time.perf_counter()
        pp = C.c_int64()
        ll = C.c_int64()
        sph._check(lib.sph_counters(h, C.byref(pp), C.byref(ll)))
        lib.sph_destroy(h)
        if r > 0:
            times.append(t1 - t0)
            pairs = pp.value
    h2d = sum(pin[k].numel() * 4 for k in pin)
    d2h = sum(o.numel() * 4 for o in out)
    return dict(s=statistics.median(times), pairs_per_step=pairs, h2d=h2d, d2h=d2h)


def run_adjoint(sph, torch, spec, steps, ckpt):
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sc = sph.scene_from(spec, stream=stream.cuda_stream)
    N = spec["n_fluid"]
    seed = np.full((N, 2), 1.0 / N, np.float32)
    sc.rollout(steps, ckpt)
    sc.adjoint(seed, None, None)  # warm-up (allocates the tape, captures the segment graphs)
    sc.rollout(steps, ckpt)
    pairs_per_step, _ = sc.counters()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sc.adjoint(seed, None, None)
    e1.record(stream)
    torch.cuda.synchronize()
    total = e0.elapsed_time(e1)
    # the adjoint sweeps alone: one more reverse pass with event nodes around them (host launched)
    sc.rollout(steps, ckpt)
    sc.profile(True)
    sc.adjoint(seed, None, None)
    torch.cuda.synchronize()
    adj_ms, adj_n = sc.timing(sph.TIMING_ADJOINT)
    info = sc.adjoint_info()
    sc.close()
    return dict(ms=total, pairs_per_step=pairs_per_step, adj_sweep_ms=adj_ms / max(adj_n, 1), adj_sweeps=adj_n,
                **info)


def _stream_specs(n_scenes: int, rate: float, seed: int = 0, skin_over_H: float = 0.0):
    """The served stream's requests; both the plain path and the server get the same scenes (with
    the same Verlet skin, a neighbour-search setting that leaves the neighbours unchanged)."""
    import sph_inputs as si
    from paper_2507_21684_b300 import tune
    reqs = si.served_stream(n_scenes=n_scenes, rate_hz=rate, seed=seed)
    out = []
    for r in reqs:
        sp = si.taylor_green_2d(r.n_side, seed=r.seed)
        if skin_over_H > 0:
            sp = tune.with_skin(sp, skin_over_H)
        out.append((r, sp))
    return out


def run_plain(sph, reqs):
    """Each request alone, in arrival order, one after another (the per-scene GPU path)."""
    import torch
    t0 = time.perf_counter()
    lat, ps = [], 0.0
    for r, sp in reqs:
        now = time.perf_counter() - t0
        if now < r.arrival_s:
            time.sleep(r.arrival_s - now)
        with sph.scene_from(sp) as sc:
            if r.adjoint:
                sc.rollout(r.steps, 20)
                x, _, _ = sc.get_state()
                seed = (2.0 * (x.astype(np.float64) - sp["x"]) / sp["n_fluid"]).astype(np.float32)
                sc.adjoint(seed, None, None)
            else:
                sc.step(r.steps)
                sc.get_state()
        lat.append(time.perf_counter() - t0 - r.arrival_s)
        ps += sp["n_fluid"] * r.steps
    span = time.perf_counter() - t0
    return dict(particle_steps_per_s=ps / span, p50_s=float(np.percentile(lat, 50)),
                p99_s=float(np.percentile(lat, 99)), makespan_s=span, _lat=lat)


def run_served(sph, reqs, budget=120 << 30, max_active=1024):
    """Requests submitted at their arrival times to the continuous-batching server (at most
    max_active requests admitted at once)."""
    with sph.Server(budget, max_active) as sv:
        t0 = time.perf_counter()
        tickets = []
        for r, sp in reqs:
            now = time.perf_counter() - t0
            if now < r.arrival_s:
                time.sleep(r.arrival_s - now)
            tickets.append((sv.submit(sp, r.steps, adjoint=r.adjoint, ckpt_every=20), r, sp))
        lat, wait, ps = [], [], 0.0
        t_end = 0.0
        for t, r, sp in tickets:
            res = sv.wait(t)
            lat.append(res["t_done"] - res["t_submit"])
            wait.append(res["t_admit"] - res["t_submit"])
            t_end = max(t_end, res["t_done"])
            ps += sp["n_fluid"] * r.steps
        span = time.perf_counter() - t0
        info = sv.stats()
    return dict(particle_steps_per_s=ps / span, p50_s=float(np.percentile(lat, 50)),
                p99_s=float(np.percentile(lat, 99)), makespan_s=span, max_batch=info["max_batch"],
                repacks=info["repacks"], _lat=lat, _wait=wait)


def latency_diag(reqs, pl, sv, top: int = 6):
    """Where the latencies differ: mean latency per request class (forward / adjoint, particle
    count below or above the median) on both paths, and the requests with the largest served
    latencies (class, size, steps, plain and served latency, the served admission wait)."""
    lp, ls, ws = pl.pop("_lat"), sv.pop("_lat"), sv.pop("_wait")
    ns = np.array([sp["n_fluid"] for _, sp in reqs])
    med = float(np.median(ns))
    cls = {}
    for k, (r, sp) in enumerate(reqs):
        key = ("adj" if r.adjoint else "fwd") + ("_large" if sp["n_fluid"] > med else "_small")
        c = cls.setdefault(key, [0, 0.0, 0.0])
        c[0] += 1
        c[1] += lp[k]
        c[2] += ls[k]
    by_class = {k: {"n": c[0], "plain_mean_s": c[1] / c[0], "served_mean_s": c[2] / c[0]} for k, c in cls.items()}
    order = np.argsort(ls)[::-1][:top]
    worst = [{"adjoint": bool(reqs[k][0].adjoint), "particles": int(ns[k]), "steps": int(reqs[k][0].steps),
              "plain_s": float(lp[k]), "served_s": float(ls[k]), "served_wait_s": float(ws[k])} for k in order]
    return {"by_class": by_class, "largest_served": worst}


def cpu_baseline(spec, budget_s: float = 15.0):
    """The FP64 oracle as it stands, on the host cores: pair interactions/s on a bounded sample
    (a short rollout of the same scene)."""
    import oracle
    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
    nf = spec["n_fluid"]
    pairs = oracle.pairs(spec["params"], spec["x"])
    pairs_fluid = int((pairs[:, 0] < nf).sum())
    oracle.rollout(spec, 2)  # first steps (thread start-up) untimed
    t0 = time.perf_counter()
    oracle.rollout(spec, 8)
    per = (time.perf_counter() - t0) / 8
    n = max(2, min(4000, int(budget_s / max(per, 1e-6))))
    t0 = time.perf_counter()
    oracle.rollout(spec, n)
    dt = time.perf_counter() - t0
    # the same oracle on one core (a shorter sample: two steps)
    oracle.set_threads(1)
    n1 = max(2, min(50, int(0.2 * budget_s / max(per * cores, 1e-6))))
    t1 = time.perf_counter()
    oracle.rollout(spec, n1)
    dt1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    return dict(value=pairs_fluid * n / dt, unit=UNIT, cores=cores, kind="oracle",
                sample=f"{spec['name']}: {n} FP64 steps from the initial state ({dt:.1f} s)",
                value_1core=pairs_fluid * n1 / dt1, sample_1core=f"{n1} FP64 steps on one core ({dt1:.1f} s)")


def cpu_adjoint_baseline(spec, steps: int, ckpt: int):
    """The FP64 oracle's reverse pass of the adjoint workload on the host cores: its forward
    rollout and reverse pass of `steps` steps, timed together, in adjoint pair interactions/s
    (pairs per step x steps / the reverse call's time)."""
    import oracle
    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
    n, d = spec["n_fluid"], spec["params"]["dim"]
    pairs = oracle.pair_count(spec["params"], spec["x"])
    xb = np.full((n, d), 1.0 / n)
    t0 = time.perf_counter()
    oracle.adjoint(spec, steps, xb, np.zeros((n, d)), np.zeros(n))
    dt = time.perf_counter() - t0
    return dict(value=pairs * steps / dt, unit="adjoint pair interactions/s", cores=cores, kind="oracle",
                s=dt, sample=f"{spec['name']}: FP64 forward + reverse pass of {steps} steps at full size "
                             f"({dt:.1f} s; the oracle keeps every step, no checkpoints)")


def oracle_leg(sph, torch, spec, steps: int, budget_1core_s: float = 8.0):
    """The FP64 oracle on the host cores beside the GPU on the same workload: `steps` oracle steps
    from the initial state, each timed (the CPU baseline), and after every step the normwise error
    of the GPU's FP32 state against the oracle's FP64 state (displacement x_n - x_0, v, rho - rho0,
    ||gpu - oracle|| / ||oracle||, and the largest elementwise error over the field's largest
    value).  One core: the oracle's rates of a sample of particles at full size."""
    import oracle
    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
    p = spec["params"]
    d, n = p["dim"], spec["n_fluid"] + spec["n_wall"]
    rho0 = float(p["rho0"])
    pairs = oracle.pair_count(p, spec["x"])
    x0 = spec["x"].astype(np.float64).reshape(n, d)
    xo, vo, ro = x0.copy(), spec["v"].astype(np.float64).reshape(n, d), spec["rho"].astype(np.float64)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sc = sph.scene_from(spec, stream=stream.cuda_stream)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    def rmax(a, b):
        return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))

    per_step, t_cpu = [], 0.0
    for k in range(steps):
        t = time.perf_counter()
        xo, vo, ro = oracle.rollout64(spec, 1, xo, vo, ro)
        t_cpu += time.perf_counter() - t
        sc.step(1)
        xg, vg, rg = sc.get_state()
        xg = xg.astype(np.float64).reshape(n, d)
        vg = vg.astype(np.float64).reshape(n, d)
        rg = rg.astype(np.float64)
        # half an ulp of the float32 output at the oracle's values: the floor no FP32 result beats
        qx = float(np.linalg.norm(np.spacing(np.abs(xo).astype(np.float32)).astype(np.float64) / 2)
                   / max(np.linalg.norm(xo - x0), 1e-300))
        per_step.append({"step": k + 1, "x_disp": rel(xg - x0, xo - x0), "v": rel(vg, vo),
                         "rho_minus_rho0": rel(rg - rho0, ro - rho0), "x_disp_max": rmax(xg - x0, xo - x0),
                         "v_max": rmax(vg, vo), "rho_minus_rho0_max": rmax(rg - rho0, ro - rho0),
                         "x_disp_f32_floor": qx})
    sc.close()
    # one core: rates of a sample of the particles (neighbour lists of the sample included)
    oracle.set_threads(1)
    m = max(1, min(n, int(n / 64)))
    who = np.linspace(0, spec["n_fluid"] - 1, m).astype(np.int32)
    t = time.perf_counter()
    oracle.rates(spec, who=who)
    t1 = time.perf_counter() - t
    oracle.set_threads(cores)
    worst = {k: max(r[k] for r in per_step) for k in ("x_disp", "v", "rho_minus_rho0")}
    cb = dict(value=pairs * steps / t_cpu, unit=UNIT, cores=cores, kind="oracle",
              sample=f"{spec['name']}: {steps} FP64 steps at full size from the initial state "
                     f"({t_cpu:.1f} s, {pairs} ordered pairs per step)",
              value_1core=pairs * (m / n) / t1,
              sample_1core=f"rates of {m} sampled particles (1/64) at full size on one core ({t1:.1f} s; "
                           f"pairs scaled from the full step's count)")
    err = {"steps": steps, "per_step": per_step, "worst": worst,
           "norm": "||gpu - oracle|| / ||oracle|| per field over all particles (x as the displacement "
                   "x_n - x_0); *_max: largest elementwise error / largest oracle value; "
                   "x_disp_f32_floor: half an ulp of float32 x over the displacement norm",
           "gpu": "FP32 (double-single x and rho)", "oracle": "FP64"}
    return cb, err


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="headline only")
    ap.add_argument("--cpu-steps", type=int, default=20,
                    help="FP64 oracle steps at full size beside the headline (CPU baseline, FP32-vs-FP64 error)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle leg of the headline")
    ap.add_argument("--profile-run", action="store_true",
                    help="forward steps of one workload only (for ncu): no extras, e2e or CPU leg")
    ap.add_argument("--workload", default="dambreak", choices=["dambreak", "tgv3d", "adjoint"],
                    help="--profile-run: dam break or 3D Taylor-Green forward steps, or the 128^2 adjoint "
                         "(200-step rollout, checkpoints every 20, then the reverse pass; --steps reverse passes)")
    ap.add_argument("--eager", action="store_true",
                    help="--profile-run: launch kernels from the host (ncu cannot profile kernel nodes of graphs "
                         "with conditional nodes); the cells are then rebuilt every step")
    ap.add_argument("--skin", type=float, default=None,
                    help="--profile-run: Verlet skin as a fraction of H (default: 0.02 dam break, 0 3D)")
    ap.add_argument("--diffusion", type=int, default=0, choices=[0, 1],
                    help="--profile-run: 0 Molteni-Colagrossi, 1 renormalised delta-SPH diffusion")
    ap.add_argument("--shift", type=float, default=0.0, help="--profile-run: particle shifting coefficient")
    ap.add_argument("--boundary", type=int, default=0, choices=[0, 1],
                    help="--profile-run (dam break): 0 Shepard wall pressure, 1 mDBC")
    ap.add_argument("--stream-scenes", type=int, default=512, help="requests of the served mixed-size stream")
    ap.add_argument("--no-tile-tune", action="store_true", help="use the default tile shape (no variant timing)")
    ap.add_argument("--variant", default="default", help="--profile-run: tile-shape variant of the library")
    ap.add_argument("--stream-rates", type=float, nargs="*", default=[20.0, 80.0, 320.0])
    ap.add_argument("--stream-max-active", type=int, default=1024,
                    help="served stream: most requests the server admits at once")
    ap.add_argument("--stream-skin", type=float, default=0.1,
                    help="Verlet skin (fraction of H) of every request of the served stream, plain and served alike")
    ap.add_argument("--stream-only", action="store_true", help="only the served stream (plain vs served)")
    args = ap.parse_args()
    ws, rank = _dist()
    import sph_inputs as si

    if args.stream_only:  # the served mixed-size stream alone (plain vs served)
        import torch  # noqa: F401  (device memory for the library's allocator hook)
        from paper_2507_21684_b300 import build as sbuild
        sbuild.build(variant=args.variant)
        import paper_2507_21684_b300 as sph
        sph.select_variant(args.variant)
        sph.use_torch_allocator()
        out = {}
        for rate in args.stream_rates:
            reqs = _stream_specs(args.stream_scenes, rate, skin_over_H=args.stream_skin)
            pl = run_plain(sph, reqs)
            sv = run_served(sph, reqs, max_active=args.stream_max_active)
            diag = latency_diag(reqs, pl, sv)
            out[f"{rate:g}_req_s"] = {"plain": pl, "served": sv,
                                      "served_over_plain_throughput": sv["particle_steps_per_s"] / pl["particle_steps_per_s"],
                                      "served_over_plain_p99": sv["p99_s"] / pl["p99_s"], "latency_diag": diag}
        print(json.dumps({"stream_only": True, "skin_over_H": args.stream_skin, "by_rate": out}))
        return

    if args.profile_run:
        import torch
        from paper_2507_21684_b300 import build as sbuild
        sbuild.build(variant=args.variant)
        import paper_2507_21684_b300 as sph
        sph.select_variant(args.variant)
        sph.use_torch_allocator()
        from paper_2507_21684_b300 import tune
        if args.workload == "adjoint":
            sa = si.adjoint_problem(128)
            sa = dict(sa, params=tune.with_skin(sa, args.skin or 0.0)["params"])
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                sc = sph.scene_from(sa, stream=stream.cuda_stream)
            seed = np.full((sa["n_fluid"], 2), 1.0 / sa["n_fluid"], np.float32)
            t0 = time.perf_counter()
            t_adj = []
            for _ in range(max(1, args.steps)):
                sc.rollout(200, 20)
                torch.cuda.synchronize()
                ta = time.perf_counter()
                sc.adjoint(seed, None, None)
                torch.cuda.synchronize()
                t_adj.append(time.perf_counter() - ta)
            sc.close()
            print(json.dumps({"profile_run": "adjoint", "skin_over_H": args.skin or 0.0, "passes": max(1, args.steps),
                              "s_per_pass": (time.perf_counter() - t0) / max(1, args.steps),
                              "adjoint_ms_min": 1e3 * min(t_adj), "adjoint_ms_median": 1e3 * statistics.median(t_adj)}))
            return
        sp = (si.dam_break(res=128, diffusion=args.diffusion, boundary=args.boundary) if args.workload == "dambreak"
              else si.taylor_green_3d(128, seed=0, diffusion=args.diffusion))
        skin = args.skin if args.skin is not None else (0.02 if args.workload == "dambreak" else 0.0)
        sp = dict(sp, params=dict(tune.with_skin(sp, skin)["params"], shift=args.shift))
        r = run_forward(sph, torch, sp, args.steps, args.warmup, args.workload == "dambreak", torch.cuda.Stream(),
                        prof_steps=0, eager=args.eager)
        print(json.dumps({"profile_run": args.workload, "diffusion": args.diffusion, "shift": args.shift,
                          "boundary": args.boundary,
                          "skin_over_H": skin,
                          "eager": args.eager,
                          "ms_per_step": sum(r["ms"]) / len(r["ms"]), "pairs_per_step": r["pairs_per_step"]}))
        return

    spec = si.taylor_green_3d(128, seed=0)
    workload = {"workload": "3D periodic Taylor-Green WCSPH, 128^3 = 2,097,152 particles in the unit cube, lattice "
                            "jittered +-0.05 dx, Wendland C2 support 2.43 dx, Tait gamma=7, c0=10, nu=0.005, "
                            "delta-SPH delta=0.1, FP32",
                "particles": spec["n_fluid"], "step": "one full SPH time step (forward only)",
                "l2": "not flushed: the state (2 x 112 MB record buffers) exceeds the 126 MB L2",
                "graph": "CUDA graph per step"}

    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(reference_arm(spec, workload, args)))
        return

    import torch
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    from paper_2507_21684_b300 import build as sbuild
    sbuild.build()
    import paper_2507_21684_b300 as sph
    from paper_2507_21684_b300 import tune

    # tile shape (targets per tile, threads per target) chosen by the library's autotuner: each
    # variant of the library times the headline scene (3D shapes) and the dam break (2D shapes) in
    # a child process; the process then loads the library built with both choices; rank 0 decides
    tiles = tiles2 = None
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    if rank == 0 and not args.no_tile_tune:
        tiles = tune.tune_tiles(spec, steps=40, warmup=10, device=dev)
        if not args.no_extras:
            tiles2 = tune.tune_tiles(tune.with_skin(si.dam_break(res=128), 0.02), steps=100, warmup=50, device=dev)
    v3 = tiles["variant"] if tiles else "default"
    v2 = tiles2["variant"] if tiles2 else "default"
    try:
        variant = sbuild.canonical(f"{v3}+{v2}")
    except ValueError:  # the two choices set the same shape: the headline's wins
        variant = v3
    variant = replica_choice(variant)
    sbuild.build(variant=variant)
    sph.select_variant(variant)
    sph.use_torch_allocator()
    stream = torch.cuda.Stream()

    # neighbour-search setting of the headline scene chosen by the library's autotuner (a Verlet
    # skin; every candidate finds the same neighbours each step)
    tuned = tune.tune_skin(spec, skins=(0.0, 0.05, 0.1, 0.15), steps=40, warmup=10)
    best_skin = replica_choice(tuned["best"]["skin_over_H"])
    spec = dict(spec, params=tune.with_skin(spec, best_skin)["params"])
    workload = dict(workload, verlet_skin_over_H=best_skin, library_variant=variant, tile_variant_3d=v3,
                    rebuild="on the device when a particle has moved skin/2 since the last build")
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass

    clk = Clocks(torch.cuda.current_device())
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk.start()
    fw = run_forward(sph, torch, spec, args.steps, args.warmup, False, stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    t_total, pairs_total = replica_reduce(sum(fw["ms"]) / 1e3, float(fw["pairs_per_step"] * args.steps),
                                          device="cuda")
    value = pairs_total / t_total
    achieved = FLOPS_PER_PAIR[3] * fw["pairs_per_step"] / (fw["sweep_ms"] / 1e3) / 1e12

    e2e = None
    if rank == 0:
        n_e2e = 200
        ee = run_e2e(sph, torch, spec, n_e2e, 2)
        e2e = {"value": ee["pairs_per_step"] * n_e2e / ee["s"], "unit": UNIT,
               "h2d_bytes_per_step": ee["h2d"] / n_e2e, "d2h_bytes_per_step": ee["d2h"] / n_e2e,
               "call": f"sph_init(host pinned) + sph_step({n_e2e}) + sph_get_state(host pinned), host wall clock "
                       f"(the workload's 200 steps)",
               "h2d_bytes_per_call": ee["h2d"], "d2h_bytes_per_call": ee["d2h"], "s_per_call": ee["s"]}
    cb, err = None, None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cb, err = oracle_leg(sph, torch, spec, args.cpu_steps)

    extras = {}
    if not args.no_extras and rank == 0:
        extras = run_extras(sph, torch, tune, args, variant, peaks, tiles2)
    if rank == 0:
        staged3 = "SPH_W3" in sbuild.variant_macros(variant) and not sbuild.variant_macros(variant)["SPH_W3"]
        sweep_kernel = "k_sweep_t" if staged3 else "k_sweep_w"
        traffic, traffic_src = stored_traffic(f"{sweep_kernel}_tgv3d_128", v3 if v3 in tune.shape_variants(3) else "default")
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload, parallelism=f"replicas x{ws}"),
            "pairs_per_step": fw["pairs_per_step"], "gpu_launches": fw["launches"],
            "rebuilds_in_timed_region": fw["rebuilds"],
            "particle_steps_per_s": spec["n_fluid"] * args.steps * ws / t_total,
            "clocks": clocks,
            "roofline": {"bound": "alu", "kernel": f"{sweep_kernel}<3> (fused rates + kick-drift)",
                         "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP32_PEAK_TFLOPS,
                         "traffic": traffic,
                         "traffic_source": (f"{traffic_src} (ncu, one launch of the same sweep kernel and tile "
                                            f"shape; this run's library variant {variant})" if traffic_src else None),
                         "flops_per_pair": FLOPS_PER_PAIR[3], "pairs_per_launch": fw["pairs_per_step"],
                         "sweep_ms_avg": fw["sweep_ms"], "sweep_launches": fw["sweep_n"],
                         "peak_source": "derived: 148 SM x 128 FP32 lanes x 2 flop x 2.032 GHz (unit counts and "
                                        "maximum SM clock; MEASURED_PEAKS has no FP32 figure)"},
            "breakdown_ms": {"sweep": fw["sweep_ms"], "rebuild_decision_and_rebuilds": fw["rebuild_ms"],
                             "step_median": statistics.median(fw["ms"]),
                             "note": "kernel classes timed by event nodes on 50 extra profiled steps"},
            "autotune": tuned["table"],
            "autotune_tiles": tiles["table"] if tiles else None,
            "e2e": e2e, "cpu_baseline": cb, "fp32_vs_fp64": err, "extras": extras,
            "hbm_peak_gbs": peaks.get("hbm_gbs"),
            # the same kernel against the memory roofline (it is not memory bound): algorithmic
            # bytes = the state read and written once (56 B per particle in 3D), and the DRAM
            # bytes of the committed ncu capture, over the kernel's mean time
            "hbm_view": hbm_view(56.0 * spec["n_fluid"], traffic, fw["sweep_ms"], peaks.get("hbm_gbs"),
                                 stored_l2_bytes(traffic_src)),
        }
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def reference_arm(spec, workload, args) -> dict:
    """The FP64 oracle as it stands on the host cores, on the headline workload: W untimed steps,
    then K timed full-size steps (fewer if they would not end within about two minutes)."""
    import oracle
    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
    p = spec["params"]
    n, d = spec["n_fluid"], p["dim"]
    pairs = oracle.pair_count(p, spec["x"])
    x, v, r = (spec["x"].astype(np.float64).reshape(n, d), spec["v"].astype(np.float64).reshape(n, d),
               spec["rho"].astype(np.float64))
    t = time.perf_counter()
    for _ in range(max(1, min(args.warmup, 2))):
        x, v, r = oracle.rollout64(spec, 1, x, v, r)
    per = (time.perf_counter() - t) / max(1, min(args.warmup, 2))
    k = max(1, min(args.steps, int(120.0 / max(per, 1e-6))))
    t = time.perf_counter()
    for _ in range(k):
        x, v, r = oracle.rollout64(spec, 1, x, v, r)
    dt = time.perf_counter() - t
    value = pairs * k / dt
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / k, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic", "config": workload,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{spec['name']}: {k} of the {args.steps} requested FP64 steps at full size "
                                       f"after {max(1, min(args.warmup, 2))} untimed ({dt:.1f} s)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_extras(sph, torch, tune, args, variant, peaks, tiles2=None) -> dict:
    """The other workloads: the dam break (and its variants), the adjoint rollout, shifting by
    optimisation, the served stream, and the oracle beside the small configurations."""
    extras = {}
    import sph_inputs as si
    # the 2D dam break (36,626 particles), L2 flushed between timed steps, with the 2D tile shape
    # tuned for it (part of the loaded library variant) and its own skin
    db = si.dam_break(res=128)
    v2 = tiles2["variant"] if tiles2 else "default"
    dtuned = tune.tune_skin(db, skins=(0.0, 0.02, 0.05, 0.1, 0.2), steps=100, warmup=100)
    dskin = dtuned["best"]["skin_over_H"]
    db = dict(db, params=tune.with_skin(db, dskin)["params"])
    dfw = run_forward(sph, torch, db, args.steps, args.warmup, True, torch.cuda.Stream())
    d = {"particles": db["n_fluid"] + db["n_wall"], "verlet_skin_over_H": dskin, "tile_variant_2d": v2,
         "library_variant": variant, "autotune_tiles": tiles2["table"] if tiles2 else None,
         "autotune_skin": dtuned["table"], "l2": "flushed (320 MB write) between timed steps"}
    td = sum(dfw["ms"]) / 1e3
    traffic, src = stored_traffic("k_walls_sweep_t_dambreak_128", v2)
    ach = FLOPS_PER_PAIR[2] * dfw["pairs_per_step"] / (dfw["sweep_ms"] / 1e3) / 1e12
    d.update({"steps": args.steps, "ms_per_step": 1e3 * td / args.steps,
              "pair_interactions_per_s": dfw["pairs_per_step"] * args.steps / td,
              "sweep_ms": dfw["sweep_ms"], "rebuild_ms": dfw["rebuild_ms"], "gpu_launches": dfw["launches"],
              "roofline": {"bound": "alu", "kernel": "k_walls_sweep_t<2> (wall pass + fused rates + kick-drift)",
                           "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                           "frac": ach / FP32_PEAK_TFLOPS, "traffic": traffic, "traffic_source": src,
                           "flops_per_pair": FLOPS_PER_PAIR[2]},
              "hbm_view": hbm_view(40.0 * (db["n_fluid"] + db["n_wall"]), traffic, dfw["sweep_ms"],
                                   peaks.get("hbm_gbs"), stored_l2_bytes(src))})
    ee = run_e2e(sph, torch, db, 2000, 2)
    d["e2e"] = {"value": ee["pairs_per_step"] * 2000 / ee["s"], "unit": UNIT, "s_per_call": ee["s"],
                "call": "sph_init(host pinned) + sph_step(2000) + sph_get_state(host pinned)"}
    d["cpu_baseline"] = cpu_baseline(dict(db, name="dambreak_128"), budget_s=10.0)
    extras["dambreak_128"] = d
    spec = db
    best_skin = dskin
    # the same dam break with the renormalised delta-SPH diffusion (one more neighbour pass)
    sr = dict(si.dam_break(res=128, diffusion=1), params=dict(spec["params"], diffusion=1))
    fr = run_forward(sph, torch, sr, args.steps, args.warmup, True, torch.cuda.Stream())
    tr = sum(fr["ms"]) / 1e3
    extras["dambreak_128_renorm"] = {
        "diffusion": "renormalised delta-SPH (kernel renormalisation L_i, Antuono psi_ij)",
        "verlet_skin_over_H": best_skin, "steps": args.steps, "ms_per_step": 1e3 * tr / args.steps,
        "pair_interactions_per_s": fr["pairs_per_step"] * args.steps / tr,
        "sweep_ms": fr["sweep_ms"], "gradient_ms": fr["gradient_ms"], "walls_ms": fr["walls_ms"],
        "l2": "flushed between timed steps"}
    # ... and with both next-row features: renormalised diffusion and particle shifting
    ss = dict(sr, params=dict(sr["params"], shift=float(np.float32(0.05))))
    fs = run_forward(sph, torch, ss, args.steps, args.warmup, True, torch.cuda.Stream())
    ts = sum(fs["ms"]) / 1e3
    extras["dambreak_128_renorm_shift"] = {
        "diffusion": "renormalised", "shift": "explicit, C = 0.05, free-surface band tangential",
        "verlet_skin_over_H": best_skin, "steps": args.steps, "ms_per_step": 1e3 * ts / args.steps,
        "pair_interactions_per_s": fs["pairs_per_step"] * args.steps / ts,
        "sweep_ms": fs["sweep_ms"], "gradient_ms": fs["gradient_ms"], "shift_ms": fs["shift_ms"],
        "rebuilds_in_timed_region": fs["rebuilds"], "l2": "flushed between timed steps"}
    # the dam break with mDBC walls (ghost nodes) in place of the Shepard wall pressure
    sm = dict(si.dam_break(res=128, boundary=1), params=dict(spec["params"], boundary=1))
    fm = run_forward(sph, torch, sm, args.steps, args.warmup, True, torch.cuda.Stream())
    tm = sum(fm["ms"]) / 1e3
    extras["dambreak_128_mdbc"] = {
        "boundary": "mDBC: first-order system at mirrored ghost nodes, pseudo-inverse",
        "verlet_skin_over_H": best_skin, "steps": args.steps, "ms_per_step": 1e3 * tm / args.steps,
        "pair_interactions_per_s": fm["pairs_per_step"] * args.steps / tm,
        "sweep_ms": fm["sweep_ms"], "mdbc_walls_ms": fm["walls_ms"], "l2": "flushed between timed steps"}
    # the dam break in summation mode: density sum of the fluid (a6), then the wall pass and
    # the sweep
    sd = dict(spec, params=dict(spec["params"], density_mode=1))
    try:
        fd = run_forward(sph, torch, sd, args.steps, args.warmup, True, torch.cuda.Stream())
        td = sum(fd["ms"]) / 1e3
        extras["dambreak_128_summation"] = {
            "density": "summation (rho_i = sum_j m_j W_ij, compensated FP32 accumulation)",
            "verlet_skin_over_H": best_skin, "steps": args.steps, "ms_per_step": 1e3 * td / args.steps,
            "pair_interactions_per_s": fd["pairs_per_step"] * args.steps / td,
            "sweep_ms": fd["sweep_ms"], "density_ms": fd["density_ms"], "walls_ms": fd["walls_ms"],
            "l2": "flushed between timed steps"}
    except sph.SphError as e:  # the scene's own error (e.g. a density outside the stable band)
        extras["dambreak_128_summation"] = {"error": str(e)}
    # the 2D Taylor-Green at 64^2 (the small configuration), 100 steps, and the oracle beside it
    s0 = si.taylor_green_2d(64, seed=0)
    f0 = run_forward(sph, torch, s0, 100, args.warmup, False, torch.cuda.Stream(), prof_steps=0)
    t0 = sum(f0["ms"]) / 1e3
    extras["tgv2d_64"] = {"particles": s0["n_fluid"], "steps": 100, "ms_per_step": 1e3 * t0 / 100,
                          "pair_interactions_per_s": f0["pairs_per_step"] * 100 / t0,
                          "cpu_baseline": cpu_baseline(dict(s0, name="tgv2d_64"), budget_s=3.0),
                          "l2": "resident (state 0.3 MB), no flush"}
    # shifting by optimisation at the paper's backward-cost size: 65,536 randomly sampled
    # particles, objective (2 passes) and its gradient (2 passes) per descent iteration
    so = si.shift_problem(256, seed=0)
    obj = dict(w_grad=1.0, w_reg=1.0, reg_fraction=0.5)
    with sph.scene_from(so) as sc:
        _, g0 = sc.shift_gradient(obj)
        step = float(5e-3 * so["dx"] / max(float(np.abs(g0).max()), 1e-30))
        sc.shift_descend(obj, 3, step)  # warm-up
        sc.profile(True)
        torch.cuda.synchronize()
        tt = time.perf_counter()
        hist = sc.shift_descend(obj, 50, step)
        t_it = (time.perf_counter() - tt) / 50
        f_ms, f_n = sc.timing(sph.TIMING_OPT_OBJECTIVE)
        b_ms, b_n = sc.timing(sph.TIMING_OPT_GRADIENT)
        r_ms, r_n = sc.timing(sph.TIMING_REBUILD)
    extras["shift_opt_64k"] = {
        "particles": so["n_fluid"], "objective": "|grad <1>|^2 + pair penalty below 0.5 dx (the paper's 2D shifting)",
        "iterations": 50, "ms_per_iteration_host": 1e3 * t_it,
        "objective_ms": f_ms / max(f_n, 1), "gradient_ms": b_ms / max(b_n, 1), "rebuild_ms": r_ms / max(r_n, 1),
        "gradient_over_objective": (b_ms / max(b_n, 1)) / max(f_ms / max(f_n, 1), 1e-12),
        "loss_first_last": [float(hist[0, 0]), float(hist[-1, 0])],
        "note": "kernel classes timed by CUDA events on the scene's stream; the host time includes one cell rebuild per iteration"}
    sa = si.adjoint_problem(128)
    for name, skin in (("adjoint_128", 0.0), ("adjoint_128_skin", 0.3)):
        spa = dict(sa, params=tune.with_skin(sa, skin)["params"])
        ad = run_adjoint(sph, torch, spa, 200, 20)
        extras[name] = {
            "particles": sa["n_fluid"], "steps": 200, "ckpt_every": 20, "verlet_skin_over_H": skin,
            "ms_total": ad["ms"],
            "adjoint_pair_interactions_per_s": ad["pairs_per_step"] * 200 / (ad["ms"] / 1e3),
            "adjoint_sweep_ms": ad["adj_sweep_ms"],
            "adjoint_sweep_pairs_per_s": ad["pairs_per_step"] / (ad["adj_sweep_ms"] / 1e3),
            "replay_rebuild_interval": ad["replay_interval"], "replay_fallbacks": ad["replay_fallbacks"],
            "note": "time of sph_adjoint: 10 segment recomputes (forward replay) + 200 adjoint sweeps, "
                    "captured graphs per segment part; with the skin the replay rebuilds every "
                    "replay_rebuild_interval steps"}
    extras["adjoint_128"]["cpu_baseline"] = cpu_adjoint_baseline(dict(sa, name="adjoint_128"), 200, 20)
    stream = {}
    for rate in args.stream_rates:
        reqs = _stream_specs(args.stream_scenes, rate, skin_over_H=args.stream_skin)
        pl = run_plain(sph, reqs)
        sv = run_served(sph, reqs, max_active=args.stream_max_active)
        diag = latency_diag(reqs, pl, sv)
        stream[f"{rate:g}_req_s"] = {"plain": pl, "served": sv,
                                     "served_over_plain_throughput": sv["particle_steps_per_s"] / pl["particle_steps_per_s"],
                                     "served_over_plain_p99": sv["p99_s"] / pl["p99_s"], "latency_diag": diag}
    extras["served_stream"] = {
        "scenes": args.stream_scenes, "sizes": "log-uniform in [1024, 262144] (square lattices)",
        "steps": "uniform in [50, 500]", "adjoint_fraction": 0.2, "arrivals": "Poisson", "by_rate": stream,
        "verlet_skin_over_H": args.stream_skin,
        "metric": "fluid particle-steps/s over the makespan; latency = completion - arrival"}
    return extras

if __name__ == "__main__":
    main()
