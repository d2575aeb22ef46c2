"""CUDA path of the mDBC wall treatment vs the FP64 oracle: the walls' densities of one step
(2D dam break, a 3D tank, an exactly linear density), rates and rollouts with mDBC walls, and
the ghost-node contract."""
import numpy as np
import pytest

import sph_inputs as si
from tests.scenes import lattice, params, scene
from tests.test_gpu_parity import check_rollout, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    from paper_2507_21684_b300 import build
    build.build()
    import paper_2507_21684_b300 as m
    return m


def _snapshot(orc, s, steps):
    xo, vo, ro = orc.rollout(s, steps)
    return dict(s, x=xo.astype(np.float32), v=vo.astype(np.float32), rho=ro.astype(np.float32))


def _tank3d(n=16, seed=0):
    """3D: a fluid block [0,1]^3 (Wendland C2, support 2.5 dx) on a floor of three wall layers,
    hydrostatic-like density increasing downwards, ghosts mirrored across z = 0."""
    dx, xf = lattice(n, 3)
    rng = np.random.default_rng(seed)
    xf = xf + rng.integers(-40, 41, xf.shape) * 2.0 ** -14
    a = (np.arange(-3, n + 3) + 0.5) * dx
    X, Y, K = np.meshgrid(a, a, np.arange(3), indexing="ij")
    xw = np.stack([X.ravel(), Y.ravel(), -(K.ravel() + 0.5) * dx], 1)
    x = np.vstack([xf, xw])
    p = params(dim=3, kernel=1, H=2.5 * dx, periodic_mask=0, box_lo=(-1, -1, -1), box_hi=(2, 2, 2),
               boundary=1, g=(0.0, 0.0, -9.81), c0=20.0, dt=1e-4)
    rho = np.ones(len(x))
    rho[: len(xf)] = 1.0 + 0.01 * (1.0 - xf[:, 2]) + 0.002 * np.sin(3 * xf[:, 0])
    s = scene(p, x, rho=rho, mass=np.full(len(x), dx ** 3), nw=len(xw))
    s["ghost"] = (xw * np.array([1.0, 1.0, -1.0])).astype(np.float32)
    return s


def _tank2d_linear(n=32, seed=1):
    dx, xf = lattice(n, 2)
    rng = np.random.default_rng(seed)
    xf = xf + rng.integers(-40, 41, xf.shape) * 2.0 ** -12
    wx = (np.arange(-4, n + 4) + 0.5) * dx
    xw = np.array([(a, -(k + 0.5) * dx) for k in range(3) for a in wx])
    x = np.vstack([xf, xw])
    b = np.array([0.125, -0.25])
    p = params(H=4 * dx, periodic_mask=0, box_lo=(-1, -1), box_hi=(2, 2), boundary=1, g=(0.0, -9.81))
    rho = np.ones(len(x))
    rho[: len(xf)] = 1.0 + xf @ b
    s = scene(p, x, rho=rho, mass=np.full(len(x), dx * dx), nw=len(xw))
    s["ghost"] = np.stack([xw[:, 0], -xw[:, 1]], 1).astype(np.float32)
    return s, b


CASES = {
    "dambreak_64": lambda orc: si.dam_break(res=64, boundary=1),
    "dambreak_128_t20": lambda orc: _snapshot(orc, si.dam_break(res=128, boundary=1), 20),
    "tank3d_16": lambda orc: _tank3d(),
}


@pytest.mark.parametrize("case", list(CASES))
def test_wall_densities_of_one_step_match_oracle(sph, orc, case):
    """The GPU sums the system in FP32 (a relative perturbation of about 1e-6 of A and b for some
    50 terms) and solves it in FP64, so the wall density may differ from the oracle's by about
    1e-6 times the condition number of the (scaled) system."""
    s = CASES[case](orc)
    with sph.scene_from(s) as sc:
        sc.step(1)
        _, _, rho = sc.get_state()
    nf = s["n_fluid"]
    d = s["params"]["dim"]
    ref, sysm = orc.mdbc(s, with_system=True)
    A = sysm[:, :16].reshape(-1, 4, 4)[:, :d + 1, :d + 1]
    cond = np.array([np.linalg.cond(a) if a[0, 0] > 0 else 1.0 for a in A])
    err = np.abs(rho[nf:].astype(np.float64) - ref)
    bound = 1e-6 * (1.0 + np.minimum(cond, 1e3)) * np.abs(ref)
    assert np.all(err <= bound), (err.max(), (err / bound).max())
    assert np.median(err) < 1e-6


def test_linear_density_exact_on_gpu_walls(sph, orc):
    s, b = _tank2d_linear()
    nf = s["n_fluid"]
    with sph.scene_from(s) as sc:
        sc.step(1)
        _, _, rho = sc.get_state()
    _, sysm = orc.mdbc(s, with_system=True)
    A = sysm[:, :16].reshape(-1, 4, 4)[:, :3, :3]
    ok = (sysm[:, 0] > 0.05) & (np.array([np.linalg.cond(a) for a in A]) < 1e2)
    xw = s["x"][nf:].astype(np.float64)
    np.testing.assert_allclose(rho[nf:][ok], 1.0 + xw[ok] @ b, rtol=0, atol=3e-6)


def test_rates_with_mdbc_walls(sph, orc):
    s = _snapshot(orc, si.dam_break(res=64, boundary=1), 20)
    with sph.scene_from(s) as sc:
        g = sc.rates()
    o = orc.rates(s)
    assert rel(g["a"], o["a"]) < 1e-5
    assert rel(g["drho"], o["drho"]) < 1e-5


ROLL = {
    "dambreak_128": lambda: si.dam_break(res=128, boundary=1),
    "dambreak_64_skin": lambda: si.dam_break(res=64, boundary=1, skin=float(np.float32(0.02 * 4 / 64)),
                                             rebuild_interval=1 << 20),
    "dambreak_64_renorm_shift": lambda: si.dam_break(res=64, boundary=1, diffusion=1, shift=0.05),
    "tank3d_16": _tank3d,
}


@pytest.mark.parametrize("case", list(ROLL))
def test_ten_step_rollout_with_mdbc(sph, orc, case):
    s = ROLL[case]()
    with sph.scene_from(s) as sc:
        sc.step(10)
        x, v, rho = sc.get_state()
    xo, vo, ro = orc.rollout(s, 10)
    check_rollout(s, 10, x, v, rho, xo, vo, ro)


def test_mdbc_needs_ghosts_and_batches_bitwise(sph):
    s = si.dam_break(res=32, boundary=1)
    sc = sph.Scene(s["params"], s["n_fluid"], s["n_wall"], s["x"], s["v"], s["rho"], s["mass"])
    with pytest.raises(Exception, match="ghost"):
        sc.step(1)
    sc.close()
    specs = [si.dam_break(res=32, boundary=1), si.dam_break(res=40, boundary=1)]
    with sph.Scene.batch(specs) as bt:
        bt.step(7)
        xb, vb, rb = bt.get_state()
        rows = list(zip(bt.first_row, bt.rows))
    for spec, (f, n) in zip(specs, rows):
        with sph.scene_from(spec) as sc:
            sc.step(7)
            x, v, r = sc.get_state()
        assert np.array_equal(x, xb[f:f + n]) and np.array_equal(v, vb[f:f + n]) and np.array_equal(r, rb[f:f + n])
