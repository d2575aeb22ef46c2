"""FP64 CPU oracle of the WCSPH step and its reverse pass (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The product library never calls it and shares no code with it.

The C++ source ``sph_oracle.cpp`` is compiled with ``-ffp-contract=off`` (no fused
multiply-add contraction, so every double operation rounds exactly as written) and OpenMP
over particles in gather form (deterministic for a fixed thread count).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "sph_oracle.cpp"
_LIB = _HERE / "libsph_oracle.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle shared library next to its source."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", str(_SRC), "-o", str(_LIB) + ".tmp"]
        subprocess.run(cmd, check=True)
        os.replace(str(_LIB) + ".tmp", _LIB)
    return _LIB


class OrcParams(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("kernel", C.c_int32), ("density_mode", C.c_int32), ("periodic_mask", C.c_int32),
        ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
        ("H", C.c_double), ("dt", C.c_double), ("rho0", C.c_double), ("c0", C.c_double),
        ("gamma", C.c_double), ("nu", C.c_double), ("delta", C.c_double), ("eps", C.c_double),
        ("g", C.c_double * 3), ("rebuild_interval", C.c_int32), ("skin", C.c_double),
        ("diffusion", C.c_int32), ("shift", C.c_double), ("boundary", C.c_int32), ("ghost", C.c_void_p),
    ]


class OrcShiftLoss(C.Structure):
    _fields_ = [
        ("w_color", C.c_double), ("w_grad", C.c_double), ("w_density", C.c_double), ("w_reg", C.c_double),
        ("reg_fraction", C.c_double), ("target_kind", C.c_int32),
        ("t_base", C.c_double), ("t_amp", C.c_double), ("t_k", C.c_double * 3), ("t_phase", C.c_double),
        ("t_lo", C.c_double), ("t_hi", C.c_double), ("t_n", C.c_double * 3), ("t_c", C.c_double),
    ]


def shift_loss(o: dict) -> OrcShiftLoss:
    r = OrcShiftLoss()
    for k in ("w_color", "w_grad", "w_density", "w_reg", "reg_fraction", "t_base", "t_amp", "t_phase",
              "t_lo", "t_hi", "t_c"):
        setattr(r, k, float(o.get(k, 0.0)))
    r.target_kind = int(o.get("target_kind", 0))
    for k in range(3):
        r.t_k[k] = float(o.get("t_k", (0.0, 0.0, 0.0))[k])
        r.t_n[k] = float(o.get("t_n", (0.0, 0.0, 0.0))[k])
    return r


def params(p: dict, scene: dict | None = None) -> OrcParams:
    """The oracle's parameters; with a scene, its mDBC ghost nodes (kept alive by the result)."""
    o = OrcParams()
    o.boundary = int(p.get("boundary", 0))
    o.ghost = None
    if scene is not None and scene.get("ghost") is not None:
        g = np.ascontiguousarray(scene["ghost"], np.float32)
        o._ghost = g
        o.ghost = g.ctypes.data
    for k in ("dim", "kernel", "density_mode", "periodic_mask", "rebuild_interval"):
        setattr(o, k, int(p[k]))
    for k in ("H", "dt", "rho0", "c0", "gamma", "nu", "delta", "eps", "skin"):
        setattr(o, k, float(p[k]))
    o.diffusion = int(p.get("diffusion", 0))
    o.shift = float(p.get("shift", 0.0))
    for k in range(3):
        o.box_lo[k] = float(p["box_lo"][k])
        o.box_hi[k] = float(p["box_hi"][k])
        o.g[k] = float(p["g"][k])
    return o


_P = C.POINTER
_d = _P(C.c_double)
_f = _P(C.c_float)
_i32 = _P(C.c_int32)
_i64 = _P(C.c_int64)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(str(_LIB))
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_kernel.argtypes = [C.c_int, C.c_int, C.c_double, _d, _d, _d, _d]
        L.orc_kernel_eval.argtypes = [_P(OrcParams), _d, _d, _d]
        L.orc_cells.argtypes = [_P(OrcParams), C.c_int, _f, _i32, _i64, _i32, _i64, C.c_int64]
        L.orc_pairs_brute.argtypes = [_P(OrcParams), C.c_int, _f, C.c_int64, _i32, _i32]
        L.orc_pairs_brute.restype = C.c_int64
        L.orc_pairs_cells.argtypes = [_P(OrcParams), C.c_int, _f, C.c_int64, _i32, _i32]
        L.orc_pairs_cells.restype = C.c_int64
        L.orc_rates.argtypes = [_P(OrcParams), C.c_int, C.c_int, _f, _f, _f, _f, C.c_int, _i32, _d, _d, _d, _d, _d]
        L.orc_rollout.argtypes = [_P(OrcParams), C.c_int, C.c_int, _f, _f, _f, _f, C.c_int, _d, _d, _d]
        L.orc_rollout64.argtypes = [_P(OrcParams), C.c_int, C.c_int, _d, _d, _d, _f, C.c_double, C.c_int,
                                    _d, _d, _d]
        L.orc_jvp.argtypes = [_P(OrcParams), C.c_int, C.c_int, _d, _d, _d, _f, C.c_double, _d, _d, _d,
                              C.c_double, C.c_int, _d, _d, _d, _d, _d, _d]
        L.orc_adjoint.argtypes = [_P(OrcParams), C.c_int, C.c_int, _d, _d, _d, _f, C.c_double, C.c_int,
                                  _d, _d, _d, _d, _d, _d, _d, _d, _d, _d]
        L.orc_sym_pinv.argtypes = [C.c_int, _d, _d]
        L.orc_renorm_gradient.argtypes = [_P(OrcParams), C.c_int, C.c_int, _f, _f, _f, _f, _d, _d]
        L.orc_shift.argtypes = [_P(OrcParams), C.c_int, C.c_int, _f, _f, _f, _f, _d, _d]
        L.orc_gen_pinv.argtypes = [C.c_int, _d, _d]
        L.orc_shift_objective.argtypes = [_P(OrcParams), C.c_int, C.c_int, _d, _f, _P(OrcShiftLoss), _d, _d, _d]
        L.orc_support.argtypes = [_P(OrcParams), C.c_int, _f, _f, _f, _d, _d, _d]
        L.orc_pairs_var.argtypes = [_P(OrcParams), C.c_int, _f, _f, C.c_int64, _i32, _i32]
        L.orc_pairs_var.restype = C.c_int64
        L.orc_mdbc.argtypes = [_P(OrcParams), C.c_int, C.c_int, _f, _f, _f, _f, _d, _d]
        _lib = L
    return _lib


def _ptr(a: np.ndarray | None, ct):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_P(ct))


def set_threads(n: int) -> int:
    return lib().orc_set_threads(int(n))


def kernel(dim: int, kern: int, q: float):
    w, w1, w2, cd = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    lib().orc_kernel(dim, kern, float(q), C.byref(w), C.byref(w1), C.byref(w2), C.byref(cd))
    return w.value, w1.value, w2.value, cd.value


def kernel_eval(p: dict, r) -> tuple[float, np.ndarray]:
    P = params(p)
    r = np.ascontiguousarray(np.asarray(r, np.float64))
    W = C.c_double()
    G = np.zeros(3)
    lib().orc_kernel_eval(C.byref(P), _ptr(r, C.c_double), C.byref(W), _ptr(G, C.c_double))
    return W.value, G[: p["dim"]].copy()


def cells(p: dict, x: np.ndarray):
    """Cells per axis, per-particle key, stable (key, id) order and CSR cell offsets."""
    P = params(p)
    x = np.ascontiguousarray(x, np.float32)
    N = x.shape[0]
    n3 = np.zeros(3, np.int32)
    key = np.zeros(N, np.int64)
    ids = np.zeros(N, np.int32)
    cap = 1 << 26
    # size the offsets from the grid first
    L = [p["box_hi"][k] - p["box_lo"][k] for k in range(p["dim"])]
    cmin = float(p["H"]) + float(p["skin"])
    nc = 1
    for Lk in L:
        nc *= max(1, int(np.floor(Lk / cmin)))
    start = np.zeros(min(cap, nc + 1), np.int64)
    rc = lib().orc_cells(C.byref(P), N, _ptr(x, C.c_float), _ptr(n3, C.c_int32), _ptr(key, C.c_int64),
                         _ptr(ids, C.c_int32), _ptr(start, C.c_int64), start.size)
    if rc != 0:
        raise ValueError(f"orc_cells failed ({rc})")
    return n3, key, ids, start


def pairs(p: dict, x: np.ndarray, brute: bool = False) -> np.ndarray:
    """Ordered neighbour pairs (i, j) as an (n, 2) int32 array sorted by (i, j)."""
    P = params(p)
    x = np.ascontiguousarray(x, np.float32)
    N = x.shape[0]
    fn = lib().orc_pairs_brute if brute else lib().orc_pairs_cells
    n = fn(C.byref(P), N, _ptr(x, C.c_float), 0, None, None)
    pi = np.zeros(n, np.int32)
    pj = np.zeros(n, np.int32)
    fn(C.byref(P), N, _ptr(x, C.c_float), n, _ptr(pi, C.c_int32), _ptr(pj, C.c_int32))
    return np.stack([pi, pj], 1)


def pair_count(p: dict, x: np.ndarray) -> int:
    """Number of ordered neighbour pairs (i != j, |r| < H) at the float32 positions x (cell search;
    the lists themselves are not returned)."""
    P = params(p)
    x = np.ascontiguousarray(x, np.float32)
    return int(lib().orc_pairs_cells(C.byref(P), x.shape[0], _ptr(x, C.c_float), 0, None, None))


def rates(scene: dict, who: np.ndarray | None = None, x=None, v=None, rho=None):
    """a, drho (and the rho, p used) of fluid particles at a float32 state."""
    p = scene["params"]
    P = params(p, scene)
    x = np.ascontiguousarray(scene["x"] if x is None else x, np.float32)
    v = np.ascontiguousarray(scene["v"] if v is None else v, np.float32)
    rho = np.ascontiguousarray(scene["rho"] if rho is None else rho, np.float32)
    m = np.ascontiguousarray(scene["mass"], np.float32)
    nf, nw, d = scene["n_fluid"], scene["n_wall"], p["dim"]
    if who is not None:
        who = np.ascontiguousarray(who, np.int32)
    M = nf if who is None else who.size
    a = np.zeros((M, d))
    dr = np.zeros(M)
    ru = np.zeros(M)
    pu = np.zeros(M)
    pw = np.zeros(max(nw, 1))
    rc = lib().orc_rates(C.byref(P), nf, nw, _ptr(x, C.c_float), _ptr(v, C.c_float), _ptr(rho, C.c_float),
                         _ptr(m, C.c_float), M, _ptr(who, C.c_int32), _ptr(a, C.c_double), _ptr(dr, C.c_double),
                         _ptr(ru, C.c_double), _ptr(pu, C.c_double), _ptr(pw, C.c_double))
    if rc != 0:
        raise ValueError("orc_rates failed")
    return dict(a=a, drho=dr, rho=ru, p=pu, p_wall=pw[:nw])


def sym_pinv(M: np.ndarray) -> np.ndarray:
    """Pseudo-inverse of a symmetric d x d matrix as the kernel renormalisation takes it."""
    M = np.asarray(M, np.float64)
    d = M.shape[0]
    A = np.zeros((3, 3))
    A[:d, :d] = M
    L = np.zeros((3, 3))
    lib().orc_sym_pinv(d, _ptr(np.ascontiguousarray(A), C.c_double), _ptr(L, C.c_double))
    return L[:d, :d].copy()


def renorm_gradient(scene: dict, x=None, v=None, rho=None, with_M: bool = False):
    """<grad rho>^L of every particle (fluid rows, then wall rows) at a float32 state."""
    p = scene["params"]
    P = params(p, scene)
    x = np.ascontiguousarray(scene["x"] if x is None else x, np.float32)
    v = np.ascontiguousarray(scene["v"] if v is None else v, np.float32)
    rho = np.ascontiguousarray(scene["rho"] if rho is None else rho, np.float32)
    m = np.ascontiguousarray(scene["mass"], np.float32)
    nf, nw, d = scene["n_fluid"], scene["n_wall"], p["dim"]
    N = nf + nw
    g = np.zeros((N, d))
    M = np.zeros((N, 3, 3)) if with_M else None
    lib().orc_renorm_gradient(C.byref(P), nf, nw, _ptr(x, C.c_float), _ptr(v, C.c_float), _ptr(rho, C.c_float),
                              _ptr(m, C.c_float), _ptr(g, C.c_double), _ptr(M, C.c_double))
    if with_M:
        return g, M[:, :d, :d].copy()
    return g


def shift(scene: dict, x=None, v=None, rho=None):
    """Particle-shifting displacements (n_fluid x dim) and lambda_i of the fluid at a float32 state."""
    p = scene["params"]
    P = params(p, scene)
    x = np.ascontiguousarray(scene["x"] if x is None else x, np.float32)
    v = np.ascontiguousarray(scene["v"] if v is None else v, np.float32)
    rho = np.ascontiguousarray(scene["rho"] if rho is None else rho, np.float32)
    m = np.ascontiguousarray(scene["mass"], np.float32)
    nf, nw, d = scene["n_fluid"], scene["n_wall"], p["dim"]
    dx = np.zeros((nf, d))
    lam = np.zeros(nf)
    lib().orc_shift(C.byref(P), nf, nw, _ptr(x, C.c_float), _ptr(v, C.c_float), _ptr(rho, C.c_float),
                    _ptr(m, C.c_float), _ptr(dx, C.c_double), _ptr(lam, C.c_double))
    return dx, lam


def gen_pinv(A: np.ndarray) -> np.ndarray:
    """Pseudo-inverse of an n x n matrix (n <= 4) as the mDBC solve takes it."""
    A = np.asarray(A, np.float64)
    n = A.shape[0]
    a = np.zeros((4, 4))
    a[:n, :n] = A
    X = np.zeros((4, 4))
    lib().orc_gen_pinv(n, _ptr(np.ascontiguousarray(a), C.c_double), _ptr(X, C.c_double))
    return X[:n, :n].copy()


def mdbc(scene: dict, x=None, v=None, rho=None, with_system: bool = False):
    """mDBC densities of the wall particles at a float32 state (scene["ghost"]: ghost nodes)."""
    p = scene["params"]
    P = params(p, scene)
    x = np.ascontiguousarray(scene["x"] if x is None else x, np.float32)
    v = np.ascontiguousarray(scene["v"] if v is None else v, np.float32)
    rho = np.ascontiguousarray(scene["rho"] if rho is None else rho, np.float32)
    m = np.ascontiguousarray(scene["mass"], np.float32)
    nf, nw = scene["n_fluid"], scene["n_wall"]
    rw = np.zeros(max(nw, 1))
    sys = np.zeros((max(nw, 1), 20)) if with_system else None
    rc = lib().orc_mdbc(C.byref(P), nf, nw, _ptr(x, C.c_float), _ptr(v, C.c_float), _ptr(rho, C.c_float),
                        _ptr(m, C.c_float), _ptr(rw, C.c_double), _ptr(sys, C.c_double))
    if rc != 0:
        raise ValueError("orc_mdbc: the scene has no ghost nodes")
    if with_system:
        return rw[:nw], sys[:nw]
    return rw[:nw]


def shift_objective(scene: dict, loss: dict, x=None, direction=None):
    """Shifting objective L at FP64 positions x (all particles; walls fixed) and, with a direction
    (n_fluid x dim), its directional derivative (forward mode)."""
    p = scene["params"]
    P = params(p, scene)
    o = shift_loss(loss)
    x = np.ascontiguousarray(scene["x"] if x is None else x, np.float64)
    m = np.ascontiguousarray(scene["mass"], np.float32)
    nf, nw = scene["n_fluid"], scene["n_wall"]
    dr = None if direction is None else np.ascontiguousarray(direction, np.float64)
    L, dL = C.c_double(), C.c_double()
    lib().orc_shift_objective(C.byref(P), nf, nw, _ptr(x, C.c_double), _ptr(m, C.c_float), C.byref(o),
                              _ptr(dr, C.c_double), C.byref(L), C.byref(dL))
    return (L.value, dL.value) if direction is not None else L.value


def shift_gradient(scene: dict, loss: dict, x=None):
    """dL/dx of the fluid particles (n_fluid x dim) by one forward-mode pass per coordinate."""
    d = scene["params"]["dim"]
    nf = scene["n_fluid"]
    x = np.ascontiguousarray(scene["x"] if x is None else x, np.float64)
    g = np.zeros((nf, d))
    e = np.zeros((nf, d))
    for i in range(nf):
        for k in range(d):
            e[i, k] = 1.0
            g[i, k] = shift_objective(scene, loss, x, e)[1]
            e[i, k] = 0.0
    return g


def support(scene: dict, h: np.ndarray):
    """Search radius, super-symmetric and gather densities with per-particle radii h (all rows)."""
    P = params(scene["params"])
    x = np.ascontiguousarray(scene["x"], np.float32)
    m = np.ascontiguousarray(np.abs(scene["mass"]), np.float32)
    h = np.ascontiguousarray(h, np.float32)
    N = x.shape[0]
    out = [np.zeros(N) for _ in range(3)]
    lib().orc_support(C.byref(P), N, _ptr(x, C.c_float), _ptr(m, C.c_float), _ptr(h, C.c_float),
                      *[_ptr(o, C.c_double) for o in out])
    return dict(search_radius=out[0], rho_super=out[1], rho_gather=out[2])


def pairs_var(scene: dict, h: np.ndarray) -> np.ndarray:
    """Ordered pairs with |x_ij| < max(h_i, h_j) (brute force), sorted by (i, j)."""
    P = params(scene["params"])
    x = np.ascontiguousarray(scene["x"], np.float32)
    h = np.ascontiguousarray(h, np.float32)
    N = x.shape[0]
    n = lib().orc_pairs_var(C.byref(P), N, _ptr(x, C.c_float), _ptr(h, C.c_float), 0, None, None)
    pi = np.zeros(n, np.int32)
    pj = np.zeros(n, np.int32)
    lib().orc_pairs_var(C.byref(P), N, _ptr(x, C.c_float), _ptr(h, C.c_float), n, _ptr(pi, C.c_int32),
                        _ptr(pj, C.c_int32))
    return np.stack([pi, pj], 1)


def rollout(scene: dict, n_steps: int, x=None, v=None, rho=None):
    """FP64 rollout from the scene's float32 state (or the given float32 arrays)."""
    p = scene["params"]
    P = params(p, scene)
    x = np.ascontiguousarray(scene["x"] if x is None else x, np.float32)
    v = np.ascontiguousarray(scene["v"] if v is None else v, np.float32)
    rho = np.ascontiguousarray(scene["rho"] if rho is None else rho, np.float32)
    m = np.ascontiguousarray(scene["mass"], np.float32)
    nf, nw, d = scene["n_fluid"], scene["n_wall"], p["dim"]
    N = nf + nw
    xo, vo, ro = np.zeros((N, d)), np.zeros((N, d)), np.zeros(N)
    lib().orc_rollout(C.byref(P), nf, nw, _ptr(x, C.c_float), _ptr(v, C.c_float), _ptr(rho, C.c_float),
                      _ptr(m, C.c_float), int(n_steps), _ptr(xo, C.c_double), _ptr(vo, C.c_double),
                      _ptr(ro, C.c_double))
    return xo, vo, ro


def rollout64(scene: dict, n_steps: int, x: np.ndarray, v: np.ndarray, rho: np.ndarray, nu: float | None = None):
    p = scene["params"]
    P = params(p, scene)
    nf, nw, d = scene["n_fluid"], scene["n_wall"], p["dim"]
    N = nf + nw
    x = np.ascontiguousarray(x, np.float64)
    v = np.ascontiguousarray(v, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    m = np.ascontiguousarray(scene["mass"], np.float32)
    nu = p["nu"] if nu is None else nu
    xo, vo, ro = np.zeros((N, d)), np.zeros((N, d)), np.zeros(N)
    lib().orc_rollout64(C.byref(P), nf, nw, _ptr(x, C.c_double), _ptr(v, C.c_double), _ptr(rho, C.c_double),
                        _ptr(m, C.c_float), float(nu), int(n_steps), _ptr(xo, C.c_double), _ptr(vo, C.c_double),
                        _ptr(ro, C.c_double))
    return xo, vo, ro


def jvp(scene: dict, n_steps: int, x, v, rho, dx, dv, drho, dnu: float = 0.0, nu: float | None = None):
    p = scene["params"]
    P = params(p, scene)
    nf, nw, d = scene["n_fluid"], scene["n_wall"], p["dim"]
    N = nf + nw
    arrs = [np.ascontiguousarray(a, np.float64) for a in (x, v, rho, dx, dv, drho)]
    m = np.ascontiguousarray(scene["mass"], np.float32)
    nu = p["nu"] if nu is None else nu
    out = [np.zeros((N, d)), np.zeros((N, d)), np.zeros(N), np.zeros((N, d)), np.zeros((N, d)), np.zeros(N)]
    if (P.diffusion == 1 and P.density_mode == 0) or P.shift > 0 or (P.boundary == 1 and nw > 0):
        raise ValueError("orc_jvp: the renormalised diffusion, particle shifting and mDBC have no tangent pass")
    lib().orc_jvp(C.byref(P), nf, nw, *[_ptr(a, C.c_double) for a in arrs[:3]], _ptr(m, C.c_float), float(nu),
                  *[_ptr(a, C.c_double) for a in arrs[3:]], float(dnu), int(n_steps),
                  *[_ptr(a, C.c_double) for a in out])
    return out


def adjoint(scene: dict, n_steps: int, xb_T, vb_T, rb_T, x=None, v=None, rho=None, nu: float | None = None):
    """Reverse pass of an n-step rollout: adjoints of (x0, v0, rho0, nu) and the final state."""
    p = scene["params"]
    P = params(p, scene)
    nf, nw, d = scene["n_fluid"], scene["n_wall"], p["dim"]
    N = nf + nw
    x = np.ascontiguousarray(scene["x"] if x is None else x, np.float64)
    v = np.ascontiguousarray(scene["v"] if v is None else v, np.float64)
    rho = np.ascontiguousarray(scene["rho"] if rho is None else rho, np.float64)
    m = np.ascontiguousarray(scene["mass"], np.float32)
    nu = p["nu"] if nu is None else nu
    ins = [np.ascontiguousarray(a, np.float64) for a in (xb_T, vb_T, rb_T)]
    xb0, vb0, rb0 = np.zeros((N, d)), np.zeros((N, d)), np.zeros(N)
    nub = C.c_double()
    xT, vT, rT = np.zeros((N, d)), np.zeros((N, d)), np.zeros(N)
    if (P.diffusion == 1 and P.density_mode == 0) or P.shift > 0:
        raise ValueError("orc_adjoint: the renormalised diffusion and particle shifting have no reverse pass")
    rc = lib().orc_adjoint(C.byref(P), nf, nw, _ptr(x, C.c_double), _ptr(v, C.c_double), _ptr(rho, C.c_double),
                           _ptr(m, C.c_float), float(nu), int(n_steps), *[_ptr(a, C.c_double) for a in ins],
                           _ptr(xb0, C.c_double), _ptr(vb0, C.c_double), _ptr(rb0, C.c_double), C.byref(nub),
                           _ptr(xT, C.c_double), _ptr(vT, C.c_double), _ptr(rT, C.c_double))
    if rc != 0:
        raise ValueError("orc_adjoint: scenes without walls only")
    return dict(xb=xb0, vb=vb0, rb=rb0, nub=nub.value, x_T=xT, v_T=vT, rho_T=rT)
