"""Oracle pins of the shifting-by-optimisation objective (the paper's differentiable particle
shifting and density-target sampling: colour field, its gradient, target density, pair
penalty) and of its forward-mode derivative."""
import numpy as np
import pytest

import sph_inputs as si
from tests.scenes import lattice, params, scene

TERMS = {
    "color": dict(w_color=1.0),
    "grad": dict(w_grad=1.0),
    "density_sin": dict(w_density=1.0, target_kind=0, t_base=1.0, t_amp=0.1, t_k=(np.pi, 2.0, 0.0), t_phase=0.3),
    "density_step": dict(w_density=1.0, target_kind=1, t_lo=0.8, t_hi=1.2, t_n=(1.0, 0.0, 0.0), t_c=0.0),
    "reg": dict(w_reg=10.0, reg_fraction=0.75),
    "all": dict(w_color=1.0, w_grad=0.3, w_density=0.5, w_reg=2.0, reg_fraction=0.75, t_base=1.0, t_amp=0.1,
                t_k=(np.pi, 0.0, 0.0)),
}


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("term", list(TERMS))
def test_forward_mode_matches_central_differences(orc, term, walls):
    s = si.shift_problem(10, seed=3, walls=walls)
    loss = TERMS[term]
    x = s["x"].astype(np.float64)
    rng = np.random.default_rng(1)
    dirn = rng.standard_normal((s["n_fluid"], 2))
    L, dL = orc.shift_objective(s, loss, x, dirn)
    assert L > 0
    h = 1e-6 * s["dx"]
    xp, xm = x.copy(), x.copy()
    xp[: s["n_fluid"]] += h * dirn
    xm[: s["n_fluid"]] -= h * dirn
    fd = (orc.shift_objective(s, loss, xp) - orc.shift_objective(s, loss, xm)) / (2 * h)
    assert abs(dL - fd) <= 1e-6 * max(abs(fd), 1e-12 * L / h), (dL, fd)


def test_density_term_uses_the_summation_density(orc):
    """rho_i of the objective (self included) equals the oracle's summation density of the step:
    with the target set to those values the density term vanishes."""
    dx, x = lattice(32, 2)  # dx = 1/32: the lattice is exact in float32
    p = params(H=4 * dx, periodic_mask=0b11, density_mode=1, nu=0.0, delta=0.0)
    s = scene(p, x, mass=np.full(len(x), dx * dx))
    rho = orc.rates(s)["rho"]
    assert np.ptp(rho) < 1e-12  # a regular lattice: one density
    L = orc.shift_objective(s, dict(w_density=1.0, target_kind=0, t_base=float(rho[0]), t_amp=0.0))
    assert L < 1e-28
    L2 = orc.shift_objective(s, dict(w_density=1.0, target_kind=0, t_base=float(rho[0]) + 1e-3, t_amp=0.0))
    assert abs(L2 - 1e-6) < 1e-12


def test_regular_lattice_is_stationary_and_gradient_free(orc):
    dx, x = lattice(16, 2)
    p = params(H=4 * dx, periodic_mask=0b11)
    s = scene(p, x, mass=np.full(len(x), dx * dx))
    assert orc.shift_objective(s, dict(w_grad=1.0)) < 1e-24  # grad 1 = 0 by symmetry
    rng = np.random.default_rng(2)
    xj = x + rng.uniform(-0.1, 0.1, x.shape) * dx  # the scale of the derivative off the lattice
    for loss in (dict(w_color=1.0), dict(w_grad=1.0), dict(w_color=1.0, w_grad=1.0)):
        dirn = rng.standard_normal((len(x), 2))
        _, dL = orc.shift_objective(s, loss, None, dirn)
        _, dLj = orc.shift_objective(s, loss, xj, dirn)
        assert abs(dL) < 1e-9 * abs(dLj), (dL, dLj)


def test_pair_penalty_closed_form_and_translation_invariance(orc):
    """One pair of a regular lattice moved to distance r < a dx: the penalty counts the pair from
    both ends, 2 w (a dx - r)^2 / n; the objective is invariant under periodic translation."""
    dx, x = lattice(16, 2)
    x = x.copy()
    r = 0.5 * dx
    x[0, 0] = x[1, 0] - r
    p = params(H=4 * dx, periodic_mask=0b11)
    s = scene(p, x, mass=np.full(len(x), dx * dx))
    a = 0.75
    L = orc.shift_objective(s, dict(w_reg=3.0, reg_fraction=a), x.astype(np.float64))
    assert abs(L - 2 * 3.0 * (a * dx - r) ** 2 / len(x)) < 1e-15
    s2 = si.shift_problem(12, seed=5)
    loss = TERMS["all"]
    L0 = orc.shift_objective(s2, dict(loss, w_density=0.0))
    xt = (s2["x"].astype(np.float64) + np.array([0.375, -0.625]) + 1.0) % 2.0 - 1.0
    L1 = orc.shift_objective(s2, dict(loss, w_density=0.0), xt)
    assert abs(L1 - L0) < 1e-12 * L0


def test_gradient_descent_lowers_the_objective(orc):
    s = si.shift_problem(8, seed=4)
    loss = dict(w_grad=1.0, w_reg=1.0, reg_fraction=0.5)
    x = s["x"].astype(np.float64)
    L = [orc.shift_objective(s, loss, x)]
    for it in range(5):
        g = orc.shift_gradient(s, loss, x)
        x = x - 1e-3 * g / max(np.abs(g).max(), 1e-30) * s["dx"]
        x = (x + 1.0) % 2.0 - 1.0
        L.append(orc.shift_objective(s, loss, x))
    assert all(b < a for a, b in zip(L, L[1:])), L
