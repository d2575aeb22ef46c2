"""Python binding of libsph_b300.so, the B300 CUDA library for the weakly-compressible SPH step
of diffSPH (Winchenbach & Thuerey, arXiv 2507.21684) and its adjoint.

This module only marshals arguments to the C ABI declared in ``include/sph.h``: every step of
the method runs in the library's CUDA kernels.  There is no CPU fallback; if the library or a
GPU is missing, the calls raise.

Inputs may be numpy arrays (host) or CUDA torch tensors (device).  Device memory of a scene is
taken from PyTorch's caching allocator once torch is imported.
"""
from __future__ import annotations

import ctypes as C
import os
from pathlib import Path

import numpy as np

__all__ = ["lib", "Params", "Scene", "Server", "SphError", "rollout_fn", "library_path"]

_HERE = Path(__file__).resolve().parent
from . import build as _build  # noqa: E402  (paths of the library variants; no compilation here)

_LIBPATH = _build.lib_path(os.environ.get("SPH_B300_VARIANT", "default"))
_lib = None

SPH_OK, SPH_EINVAL, SPH_ENOMEM, SPH_ECUDA, SPH_EUNSTABLE, SPH_ETIMEOUT, SPH_EBUSY, SPH_EINTERNAL = range(8)
_NAMES = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EUNSTABLE", 5: "ETIMEOUT", 6: "EBUSY", 7: "EINTERNAL"}

# kernel classes of sph_timing
TIMING_SWEEP, TIMING_REBUILD, TIMING_WALLS, TIMING_DENSITY, TIMING_ADJOINT, TIMING_GRADIENT, TIMING_SHIFT, \
    TIMING_OPT_OBJECTIVE, TIMING_OPT_GRADIENT = range(9)
DIFFUSION_MC, DIFFUSION_RENORM = 0, 1
BOUNDARY_SHEPARD, BOUNDARY_MDBC = 0, 1


class SphError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"SPH_{_NAMES.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("kernel", C.c_int32), ("density_mode", C.c_int32), ("periodic_mask", C.c_int32),
        ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
        ("H", C.c_float), ("dt", C.c_float), ("rho0", C.c_float), ("c0", C.c_float), ("gamma", C.c_float),
        ("nu", C.c_float), ("delta", C.c_float), ("eps", C.c_float), ("g", C.c_float * 3),
        ("rebuild_interval", C.c_int32), ("skin", C.c_float), ("diffusion", C.c_int32), ("shift", C.c_float),
        ("boundary", C.c_int32),
    ]

    @classmethod
    def from_dict(cls, p: dict) -> "Params":
        o = cls()
        for k in ("dim", "kernel", "density_mode", "periodic_mask", "rebuild_interval"):
            setattr(o, k, int(p[k]))
        for k in ("H", "dt", "rho0", "c0", "gamma", "nu", "delta", "eps", "skin"):
            setattr(o, k, float(p[k]))
        o.diffusion = int(p.get("diffusion", 0))
        o.shift = float(p.get("shift", 0.0))
        o.boundary = int(p.get("boundary", 0))
        for k in range(3):
            o.box_lo[k] = float(p["box_lo"][k])
            o.box_hi[k] = float(p["box_hi"][k])
            o.g[k] = float(p["g"][k])
        return o


class ShiftObjective(C.Structure):
    _fields_ = [("w_color", C.c_float), ("w_grad", C.c_float), ("w_density", C.c_float), ("w_reg", C.c_float),
                ("reg_fraction", C.c_float), ("target_kind", C.c_int32),
                ("t_base", C.c_float), ("t_amp", C.c_float), ("t_k", C.c_float * 3), ("t_phase", C.c_float),
                ("t_lo", C.c_float), ("t_hi", C.c_float), ("t_n", C.c_float * 3), ("t_c", C.c_float)]

    @classmethod
    def from_dict(cls, o: dict) -> "ShiftObjective":
        r = cls()
        for k in ("w_color", "w_grad", "w_density", "w_reg", "reg_fraction", "t_base", "t_amp", "t_phase",
                  "t_lo", "t_hi", "t_c"):
            setattr(r, k, float(o.get(k, 0.0)))
        r.target_kind = int(o.get("target_kind", 0))
        for k in range(3):
            r.t_k[k] = float(o.get("t_k", (0.0, 0.0, 0.0))[k])
            r.t_n[k] = float(o.get("t_n", (0.0, 0.0, 0.0))[k])
        return r


class Request(C.Structure):
    _fields_ = [("params", Params), ("n_fluid", C.c_int), ("n_wall", C.c_int),
                ("x", C.c_void_p), ("v", C.c_void_p), ("rho", C.c_void_p), ("mass", C.c_void_p),
                ("n_steps", C.c_int), ("mode", C.c_int), ("ckpt_every", C.c_int), ("x_target", C.c_void_p),
                ("ghost", C.c_void_p)]


class Result(C.Structure):
    _fields_ = [("x", C.c_void_p), ("v", C.c_void_p), ("rho", C.c_void_p),
                ("xbar0", C.c_void_p), ("vbar0", C.c_void_p), ("rhobar0", C.c_void_p),
                ("nubar", C.c_double), ("loss", C.c_double),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double)]


class ServerInfo(C.Structure):
    _fields_ = [("particle_steps_fwd", C.c_double), ("particle_steps_adj", C.c_double),
                ("queued", C.c_int), ("active", C.c_int), ("max_batch", C.c_int),
                ("bytes_in_use", C.c_size_t), ("repacks", C.c_longlong), ("iterations", C.c_longlong)]


REQ_FORWARD, REQ_ADJOINT = 0, 1

_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_hooks = None


def library_path() -> Path:
    return _LIBPATH


def select_variant(name: str) -> None:
    """Use a tile-shape variant of the library (build.VARIANTS; chosen by tune.tune_tiles).  Must be
    called before the library is first used in this process."""
    global _LIBPATH
    from . import build as _b
    name = _b.canonical(name)  # raises ValueError for an unknown part
    path = _b.lib_path(name)
    if _lib is not None and path != _LIBPATH:
        raise RuntimeError("the library is already loaded; select the variant first")
    _LIBPATH = path


def lib() -> C.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not _LIBPATH.exists():
        raise ImportError(f"{_LIBPATH} is missing: run paper_2507_21684_b300/build.py (nvcc, sm_103a)")
    L = C.CDLL(str(_LIBPATH))
    P = C.POINTER
    vp = C.c_void_p
    L.sph_abi_version.restype = C.c_int
    L.sph_last_error.restype = C.c_char_p
    L.sph_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, vp]
    L.sph_init.argtypes = [P(Params), C.c_int, C.c_int, vp, vp, vp, vp, C.c_int, vp, P(vp)]
    L.sph_init_batch.argtypes = [C.c_int, P(Params), P(C.c_int), P(C.c_int), P(vp), P(vp), P(vp), P(vp), C.c_int,
                                 vp, P(vp)]
    L.sph_batch_info.argtypes = [vp, P(C.c_int), P(C.c_int32), P(C.c_int32)]
    L.sph_step.argtypes = [vp, C.c_int]
    L.sph_get_state.argtypes = [vp, vp, vp, vp, C.c_int]
    L.sph_rates.argtypes = [vp, vp, vp, vp, C.c_int]
    L.sph_density_gradient.argtypes = [vp, vp, C.c_int]
    L.sph_set_ghosts.argtypes = [vp, vp, C.c_int]
    L.sph_set_support.argtypes = [vp, vp, C.c_int]
    L.sph_adjoint_info.argtypes = [vp, P(C.c_int32), P(C.c_int64)]
    L.sph_set_adjoint_replay.argtypes = [vp, C.c_int]
    L.sph_debug_bounded_waits.argtypes = [P(C.c_int), P(C.c_int)]
    L.sph_support_query.argtypes = [vp, vp, vp, vp, C.c_int]
    L.sph_shift_gradient.argtypes = [vp, P(ShiftObjective), vp, vp, C.c_int]
    L.sph_shift_descend.argtypes = [vp, P(ShiftObjective), C.c_int, C.c_float, vp]
    L.sph_rollout.argtypes = [vp, C.c_int, C.c_int]
    L.sph_adjoint.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, C.c_int]
    L.sph_scene_info.argtypes = [vp, P(C.c_int32), P(C.c_int32)]
    L.sph_debug_cells.argtypes = [vp, vp, vp]
    L.sph_debug_pairs.argtypes = [vp, P(C.c_int64), vp, vp, C.c_int64]
    L.sph_profile.argtypes = [vp, C.c_int]
    L.sph_timing.argtypes = [vp, C.c_int, P(C.c_double), P(C.c_int64)]
    L.sph_counters.argtypes = [vp, P(C.c_int64), P(C.c_int64)]
    L.sph_stats.argtypes = [vp, P(C.c_int64), P(C.c_int64), P(C.c_int64)]
    L.sph_set_execution.argtypes = [vp, C.c_int, C.c_int]
    L.sph_destroy.argtypes = [vp]
    L.sph_destroy.restype = None
    L.sph_server_create.argtypes = [C.c_size_t, C.c_int, P(vp)]
    L.sph_submit.argtypes = [vp, P(Request), P(C.c_uint64)]
    L.sph_poll.argtypes = [vp, C.c_uint64, P(C.c_int)]
    L.sph_wait.argtypes = [vp, C.c_uint64, C.c_int, P(Result)]
    L.sph_server_stats.argtypes = [vp, P(ServerInfo)]
    L.sph_server_destroy.argtypes = [vp]
    L.sph_server_destroy.restype = None
    L.sph_cells_noalloc.argtypes = [P(Params), vp, C.c_int32, vp, C.c_int64, vp, P(C.c_int32), vp]
    _lib = L
    return L


def _check(rc: int):
    if rc != SPH_OK:
        raise SphError(rc, lib().sph_last_error().decode(errors="replace"))


def _torch():
    import torch
    return torch


def use_torch_allocator():
    """Back the library's device allocations with PyTorch's caching allocator."""
    global _hooks
    if _hooks is not None:
        return
    torch = _torch()

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    _hooks = (_ALLOC_FN(_alloc), _FREE_FN(_free))
    _check(lib().sph_set_allocator(_hooks[0], _hooks[1], None))


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _arg(a, dtype=np.float32):
    """(pointer, keepalive, is_device) for a numpy array or a CUDA tensor."""
    if a is None:
        return None, None, None
    if _is_torch(a):
        torch = _torch()
        t = a.detach()
        if t.dtype != torch.float32:
            t = t.float()
        t = t.contiguous()
        return t.data_ptr(), t, bool(t.is_cuda)
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, arr, False


class Scene:
    """One SPH scene (or a batch of independent scenes) in HBM: initial state in, steps,
    rollouts and adjoints through the C ABI."""

    def __init__(self, params: dict, n_fluid: int, n_wall: int, x, v, rho, mass, stream=None):
        self._init_batch([params], [n_fluid], [n_wall], [x], [v], [rho], [mass], stream)

    @classmethod
    def batch(cls, specs: list, stream=None, device: bool = False) -> "Scene":
        """One scene object advancing several independent scenes with shared launches."""
        self = cls.__new__(cls)
        arr = lambda a: _torch().from_numpy(np.ascontiguousarray(a)).cuda() if device else a
        self._init_batch([s["params"] for s in specs], [s["n_fluid"] for s in specs], [s["n_wall"] for s in specs],
                         [arr(s["x"]) for s in specs], [arr(s["v"]) for s in specs], [arr(s["rho"]) for s in specs],
                         [arr(s["mass"]) for s in specs], stream)
        if any(int(s["params"].get("boundary", 0)) == BOUNDARY_MDBC and s["n_wall"] > 0 for s in specs):
            self.set_ghosts(np.concatenate([np.asarray(s["ghost"], np.float32).reshape(-1) for s in specs]))
        return self

    def _init_batch(self, params, n_fluid, n_wall, xs, vs, rhos, masses, stream):
        L = lib()
        S = len(params)
        self.n_scenes = S
        self.params = dict(params[0])
        self.dim = int(params[0]["dim"])
        self.n_fluid = int(sum(n_fluid))
        self.n_wall = int(sum(n_wall))
        self.n = self.n_fluid + self.n_wall
        keep = []
        ptrs = {k: (C.c_void_p * S)() for k in ("x", "v", "rho", "mass")}
        dev = set()
        for k in range(S):
            for name, a in (("x", xs[k]), ("v", vs[k]), ("rho", rhos[k]), ("mass", masses[k])):
                p, ref, d = _arg(a)
                ptrs[name][k] = p
                keep.append(ref)
                if d is not None:
                    dev.add(d)
        if len(dev) != 1:
            raise ValueError("inputs must be all host arrays or all CUDA tensors")
        self.device_inputs = dev.pop()
        if self.device_inputs:
            use_torch_allocator()
        if stream is None and self.device_inputs:
            stream = _torch().cuda.current_stream().cuda_stream
        self.stream = int(stream or 0)
        self._pa = (Params * S)(*[Params.from_dict(p) for p in params])
        nf = (C.c_int * S)(*[int(a) for a in n_fluid])
        nw = (C.c_int * S)(*[int(a) for a in n_wall])
        h = C.c_void_p()
        _check(L.sph_init_batch(S, self._pa, nf, nw, ptrs["x"], ptrs["v"], ptrs["rho"], ptrs["mass"],
                                int(self.device_inputs), C.c_void_p(self.stream), C.byref(h)))
        self._h = h
        first = (C.c_int32 * S)()
        rows = (C.c_int32 * S)()
        _check(L.sph_batch_info(h, None, first, rows))
        self.first_row = list(first)
        self.rows = list(rows)

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            lib().sph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- forward
    def step(self, n: int = 1):
        _check(lib().sph_step(self._h, int(n)))

    def get_state(self, device: bool = False):
        d, n = self.dim, self.n
        if device:
            torch = _torch()
            x = torch.empty((n, d), device="cuda", dtype=torch.float32)
            v = torch.empty((n, d), device="cuda", dtype=torch.float32)
            r = torch.empty((n,), device="cuda", dtype=torch.float32)
            _check(lib().sph_get_state(self._h, x.data_ptr(), v.data_ptr(), r.data_ptr(), 1))
            return x, v, r
        x = np.empty((n, d), np.float32)
        v = np.empty((n, d), np.float32)
        r = np.empty((n,), np.float32)
        _check(lib().sph_get_state(self._h, x.ctypes.data, v.ctypes.data, r.ctypes.data, 0))
        return x, v, r

    def rates(self):
        nf, d = self.n_fluid, self.dim
        a = np.empty((nf, d), np.float32)
        dr = np.empty((nf,), np.float32)
        ru = np.empty((nf,), np.float32)
        _check(lib().sph_rates(self._h, a.ctypes.data, dr.ctypes.data, ru.ctypes.data, 0))
        return dict(a=a, drho=dr, rho=ru)

    def shift_gradient(self, objective: dict):
        """Shifting objective per scene and its gradient w.r.t. every particle row (n x dim, walls 0)."""
        loss = (C.c_double * self.n_scenes)()
        g = np.empty((self.n, self.dim), np.float32)
        o = ShiftObjective.from_dict(objective)
        _check(lib().sph_shift_gradient(self._h, C.byref(o), loss, g.ctypes.data, 0))
        return np.array(loss[:]), g

    def shift_descend(self, objective: dict, n_iters: int, step: float):
        """Gradient descent on the fluid positions; the objective before each step (n_iters x scenes)."""
        hist = np.empty((int(n_iters), self.n_scenes), np.float64)
        o = ShiftObjective.from_dict(objective)
        _check(lib().sph_shift_descend(self._h, C.byref(o), int(n_iters), float(step), hist.ctypes.data))
        return hist

    def adjoint_info(self) -> dict:
        """The adjoint replay's rebuild interval and the segments that fell back to every step."""
        k, f = C.c_int32(), C.c_int64()
        _check(lib().sph_adjoint_info(self._h, C.byref(k), C.byref(f)))
        return {"replay_interval": k.value, "replay_fallbacks": f.value}

    def set_adjoint_replay(self, interval: int = 0):
        """Fix the adjoint replay's starting rebuild interval (0: from the rollout)."""
        _check(lib().sph_set_adjoint_replay(self._h, int(interval)))

    def set_support(self, H):
        """Per-particle support radii (n rows, original order), 0 < H_i <= the scene's H."""
        h = np.ascontiguousarray(np.asarray(H, np.float32).reshape(-1))
        if h.size != self.n:
            raise ValueError("one support radius per particle row")
        _check(lib().sph_set_support(self._h, h.ctypes.data, 0))

    def support_query(self):
        """Search radius, super-symmetric and gather densities of every particle row."""
        out = [np.empty(self.n, np.float32) for _ in range(3)]
        _check(lib().sph_support_query(self._h, *[o.ctypes.data for o in out], 0))
        return dict(search_radius=out[0], rho_super=out[1], rho_gather=out[2])

    def set_ghosts(self, ghost):
        """mDBC ghost nodes of the wall particles (n_wall x dim, walls in input order; a batch's
        scenes one after another)."""
        g = np.ascontiguousarray(np.asarray(ghost, np.float32).reshape(-1))
        if g.size != self.n_wall * self.dim:
            raise ValueError("ghost nodes: one per wall particle")
        _check(lib().sph_set_ghosts(self._h, g.ctypes.data, 0))

    def density_gradient(self):
        """Renormalised density gradient <grad rho>^L of every particle (n x dim, original order,
        fluid rows then wall rows), after the wall extrapolation a step applies."""
        g = np.empty((self.n, self.dim), np.float32)
        _check(lib().sph_density_gradient(self._h, g.ctypes.data, 0))
        return g

    # -- differentiation
    def rollout(self, n_steps: int, ckpt_every: int = 20):
        _check(lib().sph_rollout(self._h, int(n_steps), int(ckpt_every)))

    def adjoint(self, xb=None, vb=None, rb=None, device: bool = False):
        nf, d = self.n_fluid, self.dim
        ins = [_arg(a) for a in (xb, vb, rb)]
        flags = {f for _, _, f in ins if f is not None}
        if len(flags) > 1:
            raise ValueError("adjoint seeds must be all host or all device")
        is_dev = bool(flags.pop()) if flags else bool(device)
        nub = (C.c_double * self.n_scenes)()
        if is_dev:
            torch = _torch()
            ox = torch.empty((nf, d), device="cuda", dtype=torch.float32)
            ov = torch.empty((nf, d), device="cuda", dtype=torch.float32)
            orr = torch.empty((nf,), device="cuda", dtype=torch.float32)
            ptrs = [ox.data_ptr(), ov.data_ptr(), orr.data_ptr()]
        else:
            ox = np.empty((nf, d), np.float32)
            ov = np.empty((nf, d), np.float32)
            orr = np.empty((nf,), np.float32)
            ptrs = [ox.ctypes.data, ov.ctypes.data, orr.ctypes.data]
        _check(lib().sph_adjoint(self._h, ins[0][0], ins[1][0], ins[2][0], *ptrs, nub, int(is_dev)))
        return ox, ov, orr, (nub[0] if self.n_scenes == 1 else list(nub))

    # -- inspection
    def info(self):
        n3 = (C.c_int32 * 3)()
        n = C.c_int32()
        _check(lib().sph_scene_info(self._h, n3, C.byref(n)))
        return list(n3), n.value

    def debug_cells(self):
        n3, n = self.info()
        nc = n3[0] * n3[1] * n3[2]
        start = np.empty(nc + 1, np.int64)
        ids = np.empty(n, np.int32)
        _check(lib().sph_debug_cells(self._h, start.ctypes.data, ids.ctypes.data))
        return start, ids

    def debug_pairs(self) -> np.ndarray:
        cnt = C.c_int64()
        _check(lib().sph_debug_pairs(self._h, C.byref(cnt), None, None, 0))
        n = cnt.value
        pi = np.empty(max(n, 1), np.int32)
        pj = np.empty(max(n, 1), np.int32)
        _check(lib().sph_debug_pairs(self._h, C.byref(cnt), pi.ctypes.data, pj.ctypes.data, n))
        p = np.stack([pi[:n], pj[:n]], 1)
        order = np.lexsort((p[:, 1], p[:, 0]))
        return p[order]

    def profile(self, enable: bool = True):
        _check(lib().sph_profile(self._h, int(enable)))

    def timing(self, cls: int = TIMING_SWEEP):
        ms = C.c_double()
        n = C.c_int64()
        _check(lib().sph_timing(self._h, int(cls), C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def counters(self):
        pairs = C.c_int64()
        launches = C.c_int64()
        _check(lib().sph_counters(self._h, C.byref(pairs), C.byref(launches)))
        return pairs.value, launches.value

    def set_execution(self, use_graphs: bool = True, graph_chunk: int = 8):
        """Graph-captured chunks of steps (default) or eager launches (sph_set_execution)."""
        _check(lib().sph_set_execution(self._h, 1 if use_graphs else 0, int(graph_chunk)))

    def stats(self) -> dict:
        """Cumulative steps, cell rebuilds and kernel launches since the scene was created."""
        st, rb, ln = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().sph_stats(self._h, C.byref(st), C.byref(rb), C.byref(ln)))
        return {"steps": st.value, "rebuilds": rb.value, "launches": ln.value}


class Server:
    """Continuous-batching request loop of the library (sph_server_*)."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 256):
        h = C.c_void_p()
        _check(lib().sph_server_create(int(hbm_budget_bytes), int(max_active), C.byref(h)))
        self._h = h
        self._meta = {}

    def submit(self, spec: dict, n_steps: int, adjoint: bool = False, ckpt_every: int = 20, x_target=None) -> int:
        keep = [np.ascontiguousarray(spec[k], np.float32) for k in ("x", "v", "rho", "mass")]
        xt = None if x_target is None else np.ascontiguousarray(x_target, np.float32)
        r = Request()
        r.params = Params.from_dict(spec["params"])
        r.n_fluid, r.n_wall = int(spec["n_fluid"]), int(spec["n_wall"])
        r.x, r.v, r.rho, r.mass = (a.ctypes.data for a in keep)
        r.n_steps = int(n_steps)
        r.mode = REQ_ADJOINT if adjoint else REQ_FORWARD
        r.ckpt_every = int(ckpt_every)
        r.x_target = xt.ctypes.data if xt is not None else None
        gh = None
        if int(spec["params"].get("boundary", 0)) == BOUNDARY_MDBC and int(spec["n_wall"]) > 0:
            gh = np.ascontiguousarray(spec["ghost"], np.float32)
        r.ghost = gh.ctypes.data if gh is not None else None
        t = C.c_uint64()
        _check(lib().sph_submit(self._h, C.byref(r), C.byref(t)))
        n, d = spec["x"].shape
        self._meta[t.value] = (n, d, adjoint)
        return t.value

    def poll(self, ticket: int) -> bool:
        d = C.c_int()
        _check(lib().sph_poll(self._h, C.c_uint64(ticket), C.byref(d)))
        return bool(d.value)

    def wait(self, ticket: int, timeout_ms: int = 600000) -> dict:
        n, d, adj = self._meta[ticket]
        out = dict(x=np.empty((n, d), np.float32), v=np.empty((n, d), np.float32), rho=np.empty(n, np.float32))
        if adj:
            out.update(xbar0=np.empty((n, d), np.float32), vbar0=np.empty((n, d), np.float32),
                       rhobar0=np.empty(n, np.float32))
        r = Result()
        for k, a in out.items():
            setattr(r, k, a.ctypes.data)
        _check(lib().sph_wait(self._h, C.c_uint64(ticket), int(timeout_ms), C.byref(r)))
        del self._meta[ticket]
        out.update(nubar=r.nubar, loss=r.loss, t_submit=r.t_submit, t_admit=r.t_admit, t_done=r.t_done)
        return out

    def stats(self) -> dict:
        i = ServerInfo()
        _check(lib().sph_server_stats(self._h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in ServerInfo._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().sph_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NOALLOC_MAX_PARTICLES = 524288


def cells_noalloc(params: dict, x, cell_start, sorted_ids, stream=None) -> int:
    """Cell binning without allocation (sph_cells_noalloc): x is a contiguous CUDA float32 tensor
    (n, dim) in original order; cell_start (>= n_cells + 1 entries) and sorted_ids (>= n entries)
    are caller-owned contiguous CUDA int32 tensors that receive the CSR cell offsets and the stably
    sorted original indices (sorted_ids also serves the sort as scratch).  Work is enqueued on
    `stream` (a torch.cuda.Stream; None = the legacy default stream).  Returns n_cells.  Passing
    cell_start=None only reports n_cells (SPH_EINVAL is swallowed).  Arguments of the wrong type,
    shape or device raise ValueError before anything reaches the library."""
    dim = int(params["dim"])
    n = 0
    if x is not None:
        if not _is_torch(x) or not x.is_cuda or x.dtype != _torch().float32 or not x.is_contiguous():
            raise ValueError("cells_noalloc: x must be a contiguous CUDA float32 tensor")
        if x.dim() != 2 or int(x.shape[1]) != dim:
            raise ValueError(f"cells_noalloc: x must have shape (n, {dim}), got {tuple(x.shape)}")
        n = int(x.shape[0])
    nc = C.c_int32(0)
    st = None if stream is None else C.c_void_p(stream.cuda_stream)
    pp = Params.from_dict(params)
    if cell_start is None:
        lib().sph_cells_noalloc(C.byref(pp), None, 0, None, 0, None, C.byref(nc), st)
        return nc.value
    torch = _torch()
    for name, t in (("cell_start", cell_start), ("sorted_ids", sorted_ids)):
        if t is None and name == "sorted_ids" and n == 0:
            continue
        if not _is_torch(t) or not t.is_cuda or t.dtype != torch.int32 or not t.is_contiguous():
            raise ValueError(f"cells_noalloc: {name} must be a contiguous CUDA int32 tensor")
    lib().sph_cells_noalloc(C.byref(pp), None, 0, None, 0, None, C.byref(nc), st)
    if int(cell_start.numel()) < nc.value + 1:
        raise ValueError(f"cells_noalloc: cell_start needs n_cells + 1 = {nc.value + 1} entries, "
                         f"has {int(cell_start.numel())}")
    if n and int(sorted_ids.numel()) < n:
        raise ValueError(f"cells_noalloc: sorted_ids needs n = {n} entries, has {int(sorted_ids.numel())}")
    _check(lib().sph_cells_noalloc(C.byref(pp), x.data_ptr() if n else None, n, cell_start.data_ptr(),
                                   int(cell_start.numel()), sorted_ids.data_ptr() if n else None,
                                   C.byref(nc), st))
    return nc.value


def scene_from(spec: dict, stream=None, device: bool = False) -> Scene:
    """Scene from a generator dict (sph_inputs): host arrays, or CUDA tensors if device."""
    arrs = [spec[k] for k in ("x", "v", "rho", "mass")]
    if device:
        torch = _torch()
        arrs = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]
    sc = Scene(spec["params"], spec["n_fluid"], spec["n_wall"], *arrs, stream=stream)
    if int(spec["params"].get("boundary", 0)) == BOUNDARY_MDBC and spec["n_wall"] > 0:
        sc.set_ghosts(spec["ghost"])
    return sc


def rollout_fn():
    """torch.autograd.Function: (x0, v0, rho0, nu) -> (x_T, v_T, rho_T) through sph_rollout, with
    the backward pass through sph_adjoint (checkpoint every `ckpt_every` steps)."""
    torch = _torch()

    class SphRollout(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x0, v0, rho0, nu, mass, params, n_steps, ckpt_every):
            p = dict(params)
            p["nu"] = float(nu.detach().cpu().item()) if torch.is_tensor(nu) else float(nu)
            sc = Scene(p, x0.shape[0], 0, x0, v0, rho0, mass)
            sc.rollout(int(n_steps), int(ckpt_every))
            xT, vT, rT = sc.get_state(device=True)
            ctx.scene = sc
            return xT, vT, rT

        @staticmethod
        def backward(ctx, gx, gv, gr):
            sc = ctx.scene
            z = lambda g, shape: g.contiguous() if g is not None else torch.zeros(shape, device="cuda")
            xb, vb, rb, nub = sc.adjoint(z(gx, (sc.n, sc.dim)), z(gv, (sc.n, sc.dim)), z(gr, (sc.n,)))
            sc.close()
            ctx.scene = None
            nu_grad = torch.tensor(nub, dtype=torch.float32, device="cuda")
            return xb, vb, rb, nu_grad, None, None, None, None

    return SphRollout
