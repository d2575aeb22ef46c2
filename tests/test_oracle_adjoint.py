"""Oracle reverse pass pinned to forward-mode dual numbers (dot-product test) and to central
finite differences (Sec. 2.2: the VJP of the recurrent step composition)."""
import numpy as np
import pytest

import sph_inputs as si


def _setup(n_side=16, seed=2, density_mode=0):
    s = si.taylor_green_2d(n_side, seed=seed, density_mode=density_mode)
    N, d = s["n_fluid"], 2
    rng = np.random.default_rng(seed)
    x0 = s["x"].astype(np.float64)
    v0 = s["v"].astype(np.float64)
    r0 = s["rho"].astype(np.float64) * (1 + 0.01 * rng.standard_normal(N))
    yb = [rng.standard_normal((N, d)), rng.standard_normal((N, d)), rng.standard_normal(N)]
    tan = [1e-3 * rng.standard_normal((N, d)), rng.standard_normal((N, d)), 1e-2 * rng.standard_normal(N)]
    return s, x0, v0, r0, yb, tan


@pytest.mark.parametrize("density_mode", [0, 1])
@pytest.mark.parametrize("steps", [1, 6])
def test_vjp_matches_dual_number_jvp(orc, steps, density_mode):
    """Continuity and summation density (the latter: rho^ = sum_j m_j W_ij of the positions feeds
    the rates and is the stored density, so the position adjoint gains its chain)."""
    s, x0, v0, r0, yb, tan = _setup(density_mode=density_mode)
    dnu = 0.7
    adj = orc.adjoint(s, steps, *yb, x=x0, v=v0, rho=r0)
    out = orc.jvp(s, steps, x0, v0, r0, *tan, dnu=dnu)
    lhs = sum((a * b).sum() for a, b in zip((adj["xb"], adj["vb"], adj["rb"]), tan)) + adj["nub"] * dnu
    rhs = sum((a * b).sum() for a, b in zip(yb, out[3:]))
    assert abs(lhs - rhs) < 1e-10 * (abs(lhs) + abs(rhs))
    # the dual forward carries the same primal as the plain rollout
    xo, vo, ro = orc.rollout64(s, steps, x0, v0, r0)
    assert np.array_equal(out[0], xo) and np.array_equal(out[1], vo) and np.array_equal(out[2], ro)
    assert np.array_equal(adj["x_T"], xo)


@pytest.mark.parametrize("density_mode", [0, 1])
def test_vjp_matches_central_differences(orc, density_mode):
    s, x0, v0, r0, yb, tan = _setup(seed=5, density_mode=density_mode)
    steps = 4
    adj = orc.adjoint(s, steps, *yb, x=x0, v=v0, rho=r0)
    nu = s["params"]["nu"]

    def L(eps, dnu=0.0):
        xo, vo, ro = orc.rollout64(s, steps, x0 + eps * tan[0], v0 + eps * tan[1], r0 + eps * tan[2], nu=nu + eps * dnu)
        return (yb[0] * xo).sum() + (yb[1] * vo).sum() + (yb[2] * ro).sum()

    h = 1e-5
    fd = (L(h) - L(-h)) / (2 * h)
    an = sum((a * b).sum() for a, b in zip((adj["xb"], adj["vb"], adj["rb"]), tan))
    assert abs(fd - an) < 1e-6 * abs(an)
    fd_nu = (L(h, 1.0) - L(-h, 1.0)) / (2 * h) - fd
    assert abs(fd_nu - adj["nub"]) < 1e-5 * abs(adj["nub"]) + 1e-9


def test_loss_seed_position_mse(orc):
    """MSE of final positions against a target (Sec. 4.1 loss form): the seed is 2 (x - x~)/N."""
    s = si.taylor_green_2d(16, seed=1)
    steps = 3
    vt = si.perturbed_velocity(s)
    xt, _, _ = orc.rollout(s, steps, v=vt)
    N = s["n_fluid"]
    x0, v0, r0 = (s[k].astype(np.float64) for k in ("x", "v", "rho"))
    xo, _, _ = orc.rollout64(s, steps, x0, v0, r0)
    seed = 2.0 * (xo - xt) / N
    adj = orc.adjoint(s, steps, seed, np.zeros_like(xo), np.zeros(N), x=x0, v=v0, rho=r0)
    rng = np.random.default_rng(3)
    dv = rng.standard_normal(v0.shape)
    h = 1e-6
    def loss(vv):
        xx, _, _ = orc.rollout64(s, steps, x0, vv, r0)
        return ((xx - xt) ** 2).sum() / N
    fd = (loss(v0 + h * dv) - loss(v0 - h * dv)) / (2 * h)
    assert abs(fd - (adj["vb"] * dv).sum()) < 1e-6 * abs(fd)


def test_summation_adjoint_ignores_the_input_density_and_has_the_density_chain(orc):
    """Summation mode: the density before the first step does not influence the rollout (its
    adjoint is exactly zero), and dropping the rho^ -> x chain changes the position adjoint (the
    chain is not negligible), which central differences in x alone confirm."""
    s, x0, v0, r0, yb, tan = _setup(seed=7, density_mode=1)
    steps = 3
    adj = orc.adjoint(s, steps, *yb, x=x0, v=v0, rho=r0)
    assert np.all(adj["rb"] == 0.0)
    a1 = orc.rollout64(s, steps, x0, v0, r0)
    a2 = orc.rollout64(s, steps, x0, v0, r0 * 1.01)
    assert all(np.array_equal(p, q) for p, q in zip(a1, a2))

    def L(eps):
        xo, vo, ro = orc.rollout64(s, steps, x0 + eps * tan[0], v0, r0)
        return (yb[0] * xo).sum() + (yb[1] * vo).sum() + (yb[2] * ro).sum()
    h = 1e-6
    fd = (L(h) - L(-h)) / (2 * h)
    an = (adj["xb"] * tan[0]).sum()
    assert abs(fd - an) < 1e-6 * abs(an)
    # the same rollout in continuity mode has a different position adjoint
    sc = dict(s, params=dict(s["params"], density_mode=0))
    adj_c = orc.adjoint(sc, steps, *yb, x=x0, v=v0, rho=r0)
    assert np.linalg.norm(adj_c["xb"] - adj["xb"]) > 1e-3 * np.linalg.norm(adj["xb"])
