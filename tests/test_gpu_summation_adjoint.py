"""Adjoint in summation mode (Sec. 2.2 applied to the summation density of Sec. 2.3) on the GPU
against the FP64 oracle's reverse pass and central finite differences.

In summation mode every step recomputes rho^_i = sum_j m_j W_ij from the positions, the rates see
rho^, and rho^ is the stored density after the step; so the position adjoint carries the chain
through rho^ (an extra gathered pass after the adjoint sweep) and the initial density's adjoint is
zero.  Bars: the adjoint bar of 1e-3 (normwise relative), as for continuity mode."""
import numpy as np
import pytest

import sph_inputs as si

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def sph():
    from paper_2507_21684_b300 import build
    build.build()
    import paper_2507_21684_b300 as m
    return m


def _summation_problem(n_side, steps=200, skin_over_H=0.0):
    s = si.adjoint_problem(n_side, steps=steps)
    p = dict(s["params"], density_mode=1)
    if skin_over_H > 0:
        p = dict(p, skin=float(np.float32(skin_over_H * p["H"])), rebuild_interval=1 << 20)
    return dict(s, params=p)


def _run(sph, orc, s, steps, ckpt=20, replay=0):
    """GPU and oracle adjoints of the position-MSE loss against the perturbed-velocity target."""
    N = s["n_fluid"]
    xt, _, _ = orc.rollout(s, steps, v=s["v_target"])
    with sph.scene_from(s) as sc:
        if replay:
            sc.set_adjoint_replay(replay)
        sc.rollout(steps, ckpt)
        xT, _, _ = sc.get_state()
        seed = (2.0 * (xT.astype(np.float64) - xt) / N).astype(np.float32)
        g = sc.adjoint(seed, None, None)
    x0, v0, r0 = (s[k].astype(np.float64) for k in ("x", "v", "rho"))
    xo, _, _ = orc.rollout64(s, steps, x0, v0, r0)
    o = orc.adjoint(s, steps, 2.0 * (xo - xt) / N, np.zeros_like(xo), np.zeros(N), x=x0, v=v0, rho=r0)
    return g, o, xt


def test_summation_adjoint_matches_oracle_and_fd(sph, orc):
    """16 x 16 copy of the adjoint workload in summation mode, 200 steps, checkpoints every 20:
    the position, velocity and viscosity adjoints against the oracle's reverse pass and against
    central differences of the FP64 loss; the initial density's adjoint is zero."""
    s = _summation_problem(16)
    steps = 200
    (gx, gv, gr, gnu), o, xt = _run(sph, orc, s, steps)
    N = s["n_fluid"]
    assert rel(gv, o["vb"]) < 1e-3
    assert rel(gx, o["xb"]) < 1e-3
    assert abs(gnu - o["nub"]) < 1e-3 * abs(o["nub"])
    assert np.all(gr == 0.0)
    x0, v0, r0 = (s[k].astype(np.float64) for k in ("x", "v", "rho"))

    def loss(x, v, nu=None):
        xx, _, _ = orc.rollout64(s, steps, x, v, r0, nu=nu)
        return ((xx - xt) ** 2).sum() / N

    rng = np.random.default_rng(11)
    h = 1e-6
    for _ in range(2):
        dv = rng.standard_normal(v0.shape)
        fd = (loss(x0, v0 + h * dv) - loss(x0, v0 - h * dv)) / (2 * h)
        assert abs((gv.astype(np.float64) * dv).sum() - fd) < 1e-3 * abs(fd)
        dx = 1e-3 * rng.standard_normal(x0.shape)  # the positions' adjoint includes the rho^ chain
        fd = (loss(x0 + h * dx, v0) - loss(x0 - h * dx, v0)) / (2 * h)
        assert abs((gx.astype(np.float64) * dx).sum() - fd) < 1e-3 * abs(fd)


def test_summation_adjoint_full_size(sph, orc):
    """128 x 128 (the adjoint workload's size), 200 steps, checkpoints every 20."""
    s = _summation_problem(128)
    (gx, gv, gr, gnu), o, _ = _run(sph, orc, s, 200)
    assert rel(gv, o["vb"]) < 1e-3
    assert rel(gx, o["xb"]) < 1e-3
    assert abs(gnu - o["nub"]) < 1e-3 * abs(o["nub"])


def test_summation_adjoint_with_a_skin(sph, orc):
    """A Verlet skin: the replay rebuilds every few steps and the gradients stay the oracle's."""
    s = _summation_problem(16, skin_over_H=0.3)
    (gx, gv, gr, gnu), o, _ = _run(sph, orc, s, 200)
    assert rel(gv, o["vb"]) < 1e-3
    assert rel(gx, o["xb"]) < 1e-3


def test_summation_checkpoint_recompute_is_bitwise_store_all(sph):
    s = _summation_problem(16, steps=40)
    N = s["n_fluid"]
    rng = np.random.default_rng(2)
    seed = rng.standard_normal((N, 2)).astype(np.float32)
    out = []
    for k in (5, 40):
        with sph.scene_from(s) as sc:
            sc.rollout(40, k)
            out.append(sc.adjoint(seed, seed, np.ones(N, np.float32)))
    for a, b in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(a, b)
    assert out[0][3] == out[1][3]


def test_summation_adjoint_3d(sph, orc):
    """3D periodic Taylor-Green (Wendland C2) at 12^3, 20 steps, against the oracle."""
    s = si.taylor_green_3d(12, seed=3)
    s = dict(s, params=dict(s["params"], density_mode=1))
    N = s["n_fluid"]
    steps = 20
    rng = np.random.default_rng(4)
    yb = [rng.standard_normal((N, 3)), rng.standard_normal((N, 3)), rng.standard_normal(N)]
    with sph.scene_from(s) as sc:
        sc.rollout(steps, 5)
        gx, gv, gr, gnu = sc.adjoint(*[y.astype(np.float32) for y in yb])
    x0, v0, r0 = (s[k].astype(np.float64) for k in ("x", "v", "rho"))
    o = orc.adjoint(s, steps, *yb, x=x0, v=v0, rho=r0)
    assert rel(gv, o["vb"]) < 1e-3
    assert rel(gx, o["xb"]) < 1e-3
    assert abs(gnu - o["nub"]) < 1e-3 * abs(o["nub"])
    assert np.all(gr == 0.0)
