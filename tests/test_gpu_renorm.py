"""CUDA path of the renormalised delta-SPH diffusion vs the FP64 oracle.

The gradient pass and the sweep's renormalised term are compared with the oracle on the same
float32 inputs: single-step rates within 1e-5 (normwise relative), 10-step rollouts within
1e-3, as for the Molteni-Colagrossi form.  The gradients themselves carry the float32 rounding
of the densities (an ulp of rho over a particle spacing), so they are compared against that
floor; on an exactly representable linear density the GPU gradient is the field's slope and the
renormalised term vanishes.
"""
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


def _dyadic_block(n_side, dim, seed, jitter_units=40):
    dx, x = lattice(n_side, dim)
    rng = np.random.default_rng(seed)
    return dx, x + rng.integers(-jitter_units, jitter_units + 1, size=x.shape) * 2.0 ** -12


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_density_gradient_and_vanishing_diffusion(sph, orc, dim):
    """Free-surface block, dyadic positions and rho = 1 + b.x exact in float32, v = 0: the GPU
    gradient equals b to float32 accumulation, and the renormalised density rate vanishes while
    the Molteni-Colagrossi one does not."""
    n = 32 if dim == 2 else 16
    dx, x = _dyadic_block(n, dim, seed=7 + dim)
    H = 4 * dx if dim == 2 else 2.5 * dx
    b = np.array([0.25, -0.125, 0.0625][:dim])
    p = params(dim=dim, kernel=0 if dim == 2 else 1, H=H, periodic_mask=0, box_lo=(-1,) * dim,
               box_hi=(2,) * dim, nu=0.0, delta=0.1, diffusion=1)
    s = scene(p, x, rho=1.0 + x @ b, mass=np.full(len(x), dx ** dim))
    with sph.scene_from(s) as sc:
        g = sc.density_gradient()
        rn = sc.rates()["drho"]
    np.testing.assert_allclose(g, np.broadcast_to(b, g.shape), rtol=0, atol=2e-5 * np.abs(b).max())
    with sph.scene_from(dict(s, params=dict(p, diffusion=0))) as sc:
        mc = sc.rates()["drho"]
    assert np.abs(mc).max() > 1e-3
    assert np.abs(rn).max() < 1e-4 * np.abs(mc).max()
    # the oracle agrees on the same inputs
    assert np.abs(orc.rates(s)["drho"]).max() < 1e-10 * np.abs(mc).max()


GRAD_CASES = {
    "dambreak_64_t20": lambda orc: _snapshot(orc, si.dam_break(res=64, diffusion=1), 20),
    "tgv2d_64_pressure": lambda orc: si.taylor_green_2d(64, seed=6, pressure=True, diffusion=1),
    "tgv3d_24_pressure": lambda orc: si.taylor_green_3d(24, seed=2, pressure=True, diffusion=1),
}


@pytest.mark.parametrize("case", list(GRAD_CASES))
def test_density_gradient_matches_oracle(sph, orc, case):
    """Per particle |g_gpu - g_oracle| within 1e-3 |g| plus the rounding floor: a float32 ulp of
    rho times sum_j V_j |grad W_ij| |L_i| (the oracle's M_i gives the scale)."""
    s = GRAD_CASES[case](orc)
    with sph.scene_from(s) as sc:
        g = sc.density_gradient().astype(np.float64)
    go, M = orc.renorm_gradient(s, with_M=True)
    d = s["params"]["dim"]
    H = s["params"]["H"]
    # sum_j V_j |grad W| ~ trace(M) / (typical |r|), |r| >= H/4 for most neighbours
    Lnorm = np.array([np.linalg.norm(np.linalg.pinv(m, rcond=1e-3, hermitian=True), 2) for m in M])
    floor = 4 * 2.0 ** -23 * np.abs(s["rho"]).max() * np.trace(M, axis1=1, axis2=2) / (0.25 * H) * Lnorm
    err = np.linalg.norm(g - go, axis=1)
    bound = 1e-3 * np.linalg.norm(go, axis=1) + floor
    assert np.all(err <= bound), (err / bound).max()
    assert rel(g, go) < 2e-2


RATE_CASES = {
    "tgv2d_64_pressure_t0": lambda orc: si.taylor_green_2d(64, seed=6, pressure=True, diffusion=1),
    "dambreak_64_t20": lambda orc: _snapshot(orc, si.dam_break(res=64, diffusion=1), 20),
    "tgv3d_24_t10": lambda orc: _snapshot(orc, si.taylor_green_3d(24, seed=2, diffusion=1), 10),
}


@pytest.mark.parametrize("case", list(RATE_CASES))
def test_single_step_rates_renormalised(sph, orc, case):
    s = RATE_CASES[case](orc)
    with sph.scene_from(s) as sc:
        g = sc.rates()
    o = orc.rates(s)
    ea, ed = rel(g["a"], o["a"]), rel(g["drho"], o["drho"])
    assert ea < 1e-5, ea
    assert ed < 1e-5, ed


ROLL_CASES = {
    "dambreak_128": lambda: si.dam_break(res=128, diffusion=1),
    "tgv2d_64": lambda: si.taylor_green_2d(64, seed=0, diffusion=1),
    "tgv3d_32": lambda: si.taylor_green_3d(32, seed=1, diffusion=1),
    "dambreak_64_verlet": lambda: si.dam_break(res=64, diffusion=1, skin=float(np.float32(0.02 * 4 / 64)),
                                               rebuild_interval=1 << 20),
}


@pytest.mark.parametrize("case", list(ROLL_CASES))
def test_ten_step_rollout_renormalised(sph, orc, case):
    s = ROLL_CASES[case]()
    with sph.scene_from(s) as sc:
        sc.step(10)
        x, v, rho = sc.get_state()
    xo, vo, ro = orc.rollout(s, 10)
    check_rollout(s, 10, x, v, rho, xo, vo, ro)


def test_full_size_3d_renormalised_rates_sampled(sph, orc):
    """2,097,152-particle 3D Taylor-Green with its pressure field, renormalised diffusion: rates of
    4096 sampled particles (the oracle evaluates the gradients of their neighbours as well)."""
    s = si.taylor_green_3d(128, seed=0, pressure=True, diffusion=1)
    with sph.scene_from(s) as sc:
        g = sc.rates()
    idx = np.arange(0, s["n_fluid"], 512, dtype=np.int32)
    o = orc.rates(s, who=idx)
    assert rel(g["a"][idx], o["a"]) < 1e-5
    assert rel(g["drho"][idx], o["drho"]) < 1e-5


def test_renormalised_mode_rejects_rollout_and_mixed_batches(sph):
    s = si.taylor_green_2d(16, seed=0, diffusion=1)
    with sph.scene_from(s) as sc:
        with pytest.raises(Exception, match="renormalised"):
            sc.rollout(4, 2)
        sc.step(2)  # the forward step still runs
    with pytest.raises(Exception, match="diffusion"):
        sph.Scene.batch([s, si.taylor_green_2d(16, seed=1)])


def test_renormalised_batch_bitwise_equal_alone(sph):
    """A batch of renormalised scenes (gradient pass and sweep over all segments at once) gives
    each scene the bits it gets alone."""
    specs = [si.dam_break(res=32, diffusion=1), si.taylor_green_2d(24, seed=3, diffusion=1),
             si.dam_break(res=40, diffusion=1)]
    with sph.Scene.batch(specs) as bt:
        bt.step(9)
        xb, vb, rb = bt.get_state()
        rows = list(zip(bt.first_row, bt.rows))
    for spec, (f, n) in zip(specs, rows):
        with sph.scene_from(spec) as sc:
            sc.step(9)
            x, v, r = sc.get_state()
        assert np.array_equal(x, xb[f:f + n]) and np.array_equal(v, vb[f:f + n]) and np.array_equal(r, rb[f:f + n])
