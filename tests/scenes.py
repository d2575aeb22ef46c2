"""Small hand-built scenes for the oracle pins (lattices with prescribed fields)."""
import numpy as np

import sph_inputs as si


def params(dim=2, kernel=0, H=0.0625, dt=1e-3, c0=10.0, nu=0.01, delta=0.1, box_lo=(0, 0, 0),
           box_hi=(1, 1, 1), periodic_mask=0b11, g=(0, 0, 0), rho0=1.0, gamma=7.0, eps=0.01,
           density_mode=0, skin=0.0, rebuild_interval=1, diffusion=0, shift=0.0, boundary=0):
    f = lambda v: float(np.float32(v))
    return dict(dim=dim, kernel=kernel, density_mode=density_mode, periodic_mask=periodic_mask,
                box_lo=[float(b) for b in box_lo][:3] + [0.0] * (3 - len(box_lo)),
                box_hi=[float(b) for b in box_hi][:3] + [1.0] * (3 - len(box_hi)),
                H=f(H), dt=f(dt), rho0=f(rho0), c0=f(c0), gamma=f(gamma), nu=f(nu), delta=f(delta),
                eps=f(eps), g=[f(v) for v in g] + [0.0] * (3 - len(g)), rebuild_interval=rebuild_interval,
                skin=f(skin), diffusion=int(diffusion), shift=f(shift), boundary=int(boundary))


def lattice(n_side, dim=2, L=1.0, origin=0.0):
    dx = L / n_side
    g = np.meshgrid(*[np.arange(n_side)] * dim, indexing="ij")
    pts = np.stack([a.ravel()[::1] for a in g[::-1]], 1)  # x fastest
    return dx, origin + (pts + 0.5) * dx


def scene(p, x, v=None, rho=None, mass=None, nf=None, nw=0):
    n, d = x.shape
    v = np.zeros_like(x) if v is None else v
    rho = np.full(n, p["rho0"]) if rho is None else rho
    mass = np.full(n, 1.0) if mass is None else mass
    return dict(name="custom", params=p, n_fluid=n - nw if nf is None else nf, n_wall=nw, steps=1, seed=0,
                x=np.ascontiguousarray(x, np.float32), v=np.ascontiguousarray(v, np.float32),
                rho=np.ascontiguousarray(rho, np.float32), mass=np.ascontiguousarray(mass, np.float32))
