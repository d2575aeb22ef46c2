"""Seeded synthetic scene generators shared by the CUDA path's callers and the oracle tests.

This module holds no SPH arithmetic: it only lays particles on lattices, draws the
jitter and noise from a counter-based generator, and evaluates the initial
conditions (velocity fields, hydrostatic density) that define each workload.
Every array it returns is float32, so both the GPU library and the FP64 oracle
consume bit-identical initial states.

Workloads (the paper's own test families, Appendix E "Taylor-Green vortex" and the
dam-break tank; the sizes are the ones this project benchmarks):
  * ``taylor_green_2d``  periodic unit square, Wendland C4, support 4 dx.
  * ``taylor_green_3d``  periodic unit cube, Wendland C2, support 2.43 dx.
  * ``dam_break``        1.0 x 2.0 column in a 4.0 x 3.0 tank, three wall layers.
  * ``served_stream``    512 Taylor-Green scenes of log-uniform size with Poisson arrivals.

Random numbers: SplitMix64 (Steele, Lea, Flood 2014) applied to a counter
``(seed, stream, particle id, component)``; the top 24 bits give a float32
uniform in [0, 1).  Normals use Box-Muller on two such uniforms.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "splitmix64", "uniform24", "normal01",
    "taylor_green_2d", "taylor_green_3d", "dam_break", "perturbed_velocity",
    "served_stream", "SceneSpec",
    "KERNEL_WENDLAND4", "KERNEL_WENDLAND2", "DENSITY_CONTINUITY", "DENSITY_SUMMATION",
    "DIFFUSION_MC", "DIFFUSION_RENORM", "BOUNDARY_SHEPARD", "BOUNDARY_MDBC", "shift_problem",
]

KERNEL_WENDLAND4 = 0
KERNEL_WENDLAND2 = 1
DENSITY_CONTINUITY = 0
DENSITY_SUMMATION = 1
DIFFUSION_MC = 0        # delta-SPH diffusion in the Molteni-Colagrossi form
DIFFUSION_RENORM = 1    # with the renormalised density gradient (Antuono et al.)
BOUNDARY_SHEPARD = 0    # wall pressure by Shepard extrapolation of the fluid's, hydrostatic term
BOUNDARY_MDBC = 1       # mDBC: first-order extrapolation from ghost nodes mirrored into the fluid

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on uint64 arrays (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def _counter(seed: int, stream: int, idx: np.ndarray, comp: int) -> np.ndarray:
    base = splitmix64(np.uint64(seed) ^ (np.uint64(stream) << np.uint64(32)))
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return splitmix64(base ^ (idx * np.uint64(8) + np.uint64(comp)))


def uniform24(seed: int, stream: int, idx, comp: int) -> np.ndarray:
    """Uniform float32 in [0, 1) with 24 random bits, one per (seed, stream, idx, comp)."""
    bits = _counter(seed, stream, idx, comp) >> np.uint64(40)
    return (bits.astype(np.float64) * (1.0 / 16777216.0)).astype(np.float32)


def normal01(seed: int, stream: int, idx, comp: int) -> np.ndarray:
    """Standard normal (float64) by Box-Muller from two counter uniforms."""
    u1 = uniform24(seed, stream, idx, 2 * comp).astype(np.float64)
    u2 = uniform24(seed, stream, idx, 2 * comp + 1).astype(np.float64)
    u1 = 1.0 - u1  # (0, 1]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def _f32(v: float) -> float:
    return float(np.float32(v))


def _params(dim, kernel, H, dt, c0, nu, delta, box_lo, box_hi, periodic_mask,
            g=(0.0, 0.0, 0.0), rho0=1.0, gamma=7.0, eps=0.01, density_mode=DENSITY_CONTINUITY,
            rebuild_interval=1, skin=0.0, diffusion=DIFFUSION_MC, shift=0.0, boundary=BOUNDARY_SHEPARD):
    return dict(
        dim=int(dim), kernel=int(kernel), density_mode=int(density_mode),
        periodic_mask=int(periodic_mask),
        box_lo=[float(b) for b in box_lo] + [0.0] * (3 - len(box_lo)),
        box_hi=[float(b) for b in box_hi] + [1.0] * (3 - len(box_hi)),
        H=_f32(H), dt=_f32(dt), rho0=_f32(rho0), c0=_f32(c0), gamma=_f32(gamma),
        nu=_f32(nu), delta=_f32(delta), eps=_f32(eps),
        g=[_f32(x) for x in g] + [0.0] * (3 - len(g)),
        rebuild_interval=int(rebuild_interval), skin=_f32(skin), diffusion=int(diffusion),
        shift=_f32(shift), boundary=int(boundary),
    )


def _lattice_2d(n_side: int, seed: int, jitter: float, L: float = 1.0):
    dx = L / n_side
    ids = np.arange(n_side * n_side, dtype=np.int64)
    ix = (ids % n_side).astype(np.float64)
    iy = (ids // n_side).astype(np.float64)
    jx = uniform24(seed, 0, ids, 0).astype(np.float64) - 0.5
    jy = uniform24(seed, 0, ids, 1).astype(np.float64) - 0.5
    x = (ix + 0.5 + 2.0 * jitter * jx) * dx
    y = (iy + 0.5 + 2.0 * jitter * jy) * dx
    return dx, np.stack([x, y], axis=1)


def _tait_inverse(p, rho0, c0, gamma):
    B = rho0 * c0 * c0 / gamma
    return rho0 * (1.0 + p / B) ** (1.0 / gamma)


def taylor_green_2d(n_side: int = 64, seed: int = 0, steps: int = 100, nu: float = 0.01,
                    c0: float = 10.0, delta: float = 0.1, jitter: float = 0.05,
                    density_mode: int = DENSITY_CONTINUITY, rebuild_interval: int = 1,
                    skin: float = 0.0, dt: float | None = None, pressure: bool = False,
                    diffusion: int = 0, shift: float = 0.0) -> dict:
    """Periodic 2D Taylor-Green vortex on the unit square (u = sin 2pi x cos 2pi y,
    v = -cos 2pi x sin 2pi y), lattice at (i+1/2)dx jittered by U[-jitter, jitter) dx,
    rho = rho0 = 1, m = rho0 dx^2, Wendland C4 with support H = 4 dx, dt = h / (4 c0) with the
    smoothing length h = H/2 unless given.  With ``pressure`` the density carries the vortex's analytic pressure
    p = (rho0 U^2 / 4)(cos 4pi x + cos 4pi y) through the inverse Tait law."""
    dx, xy = _lattice_2d(n_side, seed, jitter)
    vx = np.sin(2 * np.pi * xy[:, 0]) * np.cos(2 * np.pi * xy[:, 1])
    vy = -np.cos(2 * np.pi * xy[:, 0]) * np.sin(2 * np.pi * xy[:, 1])
    n = n_side * n_side
    H = 4.0 * dx
    dt = 0.25 * (0.5 * _f32(H)) / c0 if dt is None else dt
    p = _params(2, KERNEL_WENDLAND4, H, dt, c0, nu, delta, (0.0, 0.0), (1.0, 1.0), 0b11,
                density_mode=density_mode, rebuild_interval=rebuild_interval, skin=skin,
                diffusion=diffusion, shift=shift)
    rho = np.full(n, p["rho0"])
    if pressure:
        pr = 0.25 * (np.cos(4 * np.pi * xy[:, 0]) + np.cos(4 * np.pi * xy[:, 1]))
        rho = _tait_inverse(pr, 1.0, p["c0"], p["gamma"])
    return dict(
        name=f"tgv2d_{n_side}", params=p, n_fluid=n, n_wall=0, steps=steps, seed=seed, dx=dx,
        x=xy.astype(np.float32), v=np.stack([vx, vy], 1).astype(np.float32),
        rho=rho.astype(np.float32), mass=np.full(n, _f32(dx * dx), np.float32),
    )


def taylor_green_3d(n_side: int = 128, seed: int = 0, steps: int = 200, nu: float = 0.005,
                    c0: float = 10.0, delta: float = 0.1, jitter: float = 0.05,
                    support: float = 2.43, rebuild_interval: int = 1, skin: float = 0.0,
                    pressure: bool = False, diffusion: int = 0, shift: float = 0.0) -> dict:
    """Periodic 3D Taylor-Green vortex in the unit cube (u = sin cos cos, v = -cos sin cos,
    w = 0), Wendland C2 with support 2.43 dx, lattice jittered by U[-jitter, jitter) dx.  With
    ``pressure`` the density carries the analytic pressure
    p = (rho0 U^2 / 16)(cos 4pi x + cos 4pi y)(cos 4pi z + 2) through the inverse Tait law."""
    dx = 1.0 / n_side
    n = n_side ** 3
    ids = np.arange(n, dtype=np.int64)
    ijk = np.stack([ids % n_side, (ids // n_side) % n_side, ids // (n_side * n_side)], 1).astype(np.float64)
    jit = np.stack([uniform24(seed, 0, ids, a).astype(np.float64) - 0.5 for a in range(3)], 1)
    x = (ijk + 0.5 + 2.0 * jitter * jit) * dx
    sx, sy, sz = (np.sin(2 * np.pi * x[:, a]) for a in range(3))
    cx, cy, cz = (np.cos(2 * np.pi * x[:, a]) for a in range(3))
    v = np.stack([sx * cy * cz, -cx * sy * cz, np.zeros(n)], 1)
    H = support * dx
    p = _params(3, KERNEL_WENDLAND2, H, 0.25 * (0.5 * _f32(H)) / c0, c0, nu, delta, (0.0, 0.0, 0.0),
                (1.0, 1.0, 1.0), 0b111, rebuild_interval=rebuild_interval, skin=skin, diffusion=diffusion,
                shift=shift)
    rho = np.full(n, p["rho0"])
    if pressure:
        pr = (1.0 / 16.0) * (np.cos(4 * np.pi * x[:, 0]) + np.cos(4 * np.pi * x[:, 1])) * \
            (np.cos(4 * np.pi * x[:, 2]) + 2.0)
        rho = _tait_inverse(pr, 1.0, p["c0"], p["gamma"])
    return dict(
        name=f"tgv3d_{n_side}", params=p, n_fluid=n, n_wall=0, steps=steps, seed=seed, dx=dx,
        x=x.astype(np.float32), v=v.astype(np.float32),
        rho=rho.astype(np.float32), mass=np.full(n, _f32(dx ** 3), np.float32),
    )


def dam_break(res: int = 128, steps: int = 2000, alpha_visc: float = 0.02, delta: float = 0.1,
              rebuild_interval: int = 1, skin: float = 0.0, diffusion: int = 0, shift: float = 0.0,
              boundary: int = 0) -> dict:
    """2D dam break: fluid column [0,1] x [0,2] at (i+1/2)dx in the tank [0,4] x [0,3],
    dx = 1/res, three layers of fixed wall particles at -(k+1/2)dx (left, bottom, corners
    filled) and 4+(k+1/2)dx (right), open top.  g = (0, -9.81), c0 = 10 sqrt(2 g 2.0),
    Wendland C4 support 4 dx, hydrostatic initial density by the inverse Tait law.
    The viscosity is the delta-SPH artificial viscosity alpha = 0.02 expressed as
    nu = alpha h c0 / (2 (d + 2)) with h = H/2.  The time step is dt = dx / (4 c0) = h / (8 c0):
    with a free surface, the symplectic-Euler step at h / (4 c0) grows particle-scale modes
    within a few hundred steps (the FP64 reference diverges too), at h / (8 c0) it does not."""
    dx = 1.0 / res
    g = 9.81
    rho0 = 1.0
    gamma = 7.0
    c0 = 10.0 * math.sqrt(2.0 * g * 2.0)
    H = 4.0 * dx
    nu = alpha_visc * (0.5 * H) * c0 / (2.0 * (2 + 2))
    nfx, nfy = int(round(1.0 * res)), int(round(2.0 * res))
    fi = np.arange(nfx * nfy)
    fx = ((fi % nfx) + 0.5) * dx
    fy = ((fi // nfx) + 0.5) * dx
    # walls: bottom rows (with corners), then left and right columns up to y = 3
    nwx = int(round(4.0 * res))
    nwy = int(round(3.0 * res))
    walls = []
    for k in range(3):
        for i in range(-3, nwx + 3):
            walls.append(((i + 0.5) * dx, -(k + 0.5) * dx))
    for k in range(3):
        for j in range(nwy):
            walls.append((-(k + 0.5) * dx, (j + 0.5) * dx))
            walls.append((4.0 + (k + 0.5) * dx, (j + 0.5) * dx))
    w = np.array(walls, np.float64)
    B = rho0 * c0 * c0 / gamma
    rho_f = rho0 * (1.0 + rho0 * g * (2.0 - fy) / B) ** (1.0 / gamma)
    x = np.concatenate([np.stack([fx, fy], 1), w], 0)
    nf, nw = nfx * nfy, len(w)
    v = np.zeros((nf + nw, 2))
    rho = np.concatenate([rho_f, np.full(nw, rho0)])
    p = _params(2, KERNEL_WENDLAND4, H, 0.25 * dx / _f32(c0), c0, nu, delta,
                (-4 * dx, -4 * dx), (4.0 + 4 * dx, 3.0), 0b00, g=(0.0, -g), rho0=rho0, gamma=gamma,
                rebuild_interval=rebuild_interval, skin=skin, diffusion=diffusion, shift=shift,
                boundary=boundary)
    # mDBC ghost nodes: each wall particle mirrored across the tank's wall surfaces (x = 0, x = 4,
    # y = 0; the corner particles across both)
    gx = np.where(w[:, 0] < 0.0, -w[:, 0], np.where(w[:, 0] > 4.0, 8.0 - w[:, 0], w[:, 0]))
    gy = np.where(w[:, 1] < 0.0, -w[:, 1], w[:, 1])
    return dict(
        ghost=np.stack([gx, gy], 1).astype(np.float32),
        name=f"dambreak_{res}", params=p, n_fluid=nf, n_wall=nw, steps=steps, seed=0, dx=dx,
        x=x.astype(np.float32), v=v.astype(np.float32), rho=rho.astype(np.float32),
        mass=np.full(nf + nw, _f32(rho0 * dx * dx), np.float32),
    )


def adjoint_problem(n_side: int = 128, steps: int = 200, seed: int = 0) -> dict:
    """Adjoint workload: periodic Taylor-Green at n_side^2 with the time step of the 128^2 case
    (dt = h_128 / (4 c0) = 3.90625e-4, so the 16^2 copy covers the same 200 steps and horizon),
    target rollout from velocities perturbed by 5% Gaussian noise."""
    dt = 0.25 * (0.5 * _f32(4.0 / 128.0)) / 10.0
    s = taylor_green_2d(n_side, seed=seed, steps=steps, dt=dt)
    s["v_target"] = perturbed_velocity(s)
    s["ckpt_every"] = 20
    return s


def perturbed_velocity(scene: dict, rel: float = 0.05, U0: float = 1.0, seed: int | None = None) -> np.ndarray:
    """Initial velocities of the target rollout: v0 + rel * U0 * xi, xi ~ N(0, 1) per component."""
    seed = scene["seed"] if seed is None else seed
    n, d = scene["v"].shape
    ids = np.arange(n, dtype=np.int64)
    xi = np.stack([normal01(seed, 7, ids, a) for a in range(d)], 1)
    return (scene["v"].astype(np.float64) + rel * U0 * xi).astype(np.float32)


@dataclass
class SceneSpec:
    """One request of the served stream."""
    index: int
    n_side: int
    steps: int
    adjoint: bool
    arrival_s: float
    seed: int = field(default=0)

    @property
    def n(self) -> int:
        return self.n_side * self.n_side


def served_stream(n_scenes: int = 512, rate_hz: float = 80.0, seed: int = 0, n_min: int = 1024,
                  n_max: int = 262144, steps_lo: int = 50, steps_hi: int = 500,
                  adjoint_frac: float = 0.2) -> list[SceneSpec]:
    """Mixed-size request stream: particle counts log-uniform in [n_min, n_max] (rounded to a
    square lattice), steps uniform in [steps_lo, steps_hi], a fraction of adjoint rollouts,
    Poisson arrivals at ``rate_hz``."""
    ids = np.arange(n_scenes, dtype=np.int64)
    u_n = uniform24(seed, 11, ids, 0).astype(np.float64)
    u_s = uniform24(seed, 11, ids, 1).astype(np.float64)
    u_a = uniform24(seed, 11, ids, 2).astype(np.float64)
    u_t = uniform24(seed, 11, ids, 3).astype(np.float64)
    lo, hi = math.log(math.sqrt(n_min)), math.log(math.sqrt(n_max))
    n_side = np.rint(np.exp(lo + (hi - lo) * u_n)).astype(np.int64)
    steps = steps_lo + np.floor(u_s * (steps_hi - steps_lo + 1)).astype(np.int64)
    adj = u_a < adjoint_frac
    gaps = -np.log(1.0 - u_t) / rate_hz
    t = np.cumsum(gaps) - gaps[0]
    return [SceneSpec(int(i), int(n_side[i]), int(steps[i]), bool(adj[i]), float(t[i]), seed=int(i))
            for i in range(n_scenes)]


def shift_problem(n_side: int = 32, seed: int = 0, dim: int = 2, walls: bool = False,
                  support: float = 4.0) -> dict:
    """The paper's differentiable-shifting setup: n_side^d particles of equal mass sampled uniformly
    at random in [-1, 1]^d (rho0 = 1, m = 2^d / n), Wendland C4 (2D) or C2 (3D) with support
    `support` x the mean spacing.  Periodic, or with three layers of fixed wall particles on a
    regular lattice around the box (`walls`)."""
    n = n_side ** dim
    dx = 2.0 / n_side
    ids = np.arange(n, dtype=np.int64)
    u = np.stack([uniform24(seed, 7, ids, a).astype(np.float64) for a in range(dim)], 1)
    xf = -1.0 + 2.0 * u
    H = support * dx
    if walls:
        g = np.arange(-3, n_side + 3)
        grids = np.meshgrid(*[g] * dim, indexing="ij")
        pts = np.stack([a.ravel() for a in grids[::-1]], 1)
        xw = -1.0 + (pts + 0.5) * dx
        outside = np.any((xw < -1.0) | (xw > 1.0), axis=1)
        xw = xw[outside]
        lo, hi, mask = [-1.0 - 4 * dx] * dim, [1.0 + 4 * dx] * dim, 0
    else:
        xw = np.zeros((0, dim))
        lo, hi, mask = [-1.0] * dim, [1.0] * dim, (1 << dim) - 1
    x = np.concatenate([xf, xw], 0)
    p = _params(dim, KERNEL_WENDLAND4 if dim == 2 else KERNEL_WENDLAND2, H, 1e-3, 10.0, 0.0, 0.0,
                tuple(lo), tuple(hi), mask)
    N = len(x)
    return dict(
        name=f"shift{dim}d_{n_side}{'_walls' if walls else ''}", params=p, n_fluid=n, n_wall=len(xw), steps=1,
        seed=seed, dx=dx, x=x.astype(np.float32), v=np.zeros((N, dim), np.float32),
        rho=np.ones(N, np.float32), mass=np.full(N, _f32(dx ** dim), np.float32),
    )
