"""CUDA path of the shifting-by-optimisation objective (four gathered passes: density, colour
field and seeds, first adjoint gather, second adjoint gather with the descent step) against the
FP64 oracle: the objective within 1e-5, its gradient within 1e-3 (the adjoint bar) element by
element against the oracle's forward-mode gradient, and at full size along random directions."""
import numpy as np
import pytest

import sph_inputs as si
from tests.test_gpu_parity import rel

pytestmark = pytest.mark.gpu

TERMS = {
    "color": dict(w_color=1.0),
    "grad": dict(w_grad=1.0),
    "density_sin": dict(w_density=1.0, target_kind=0, t_base=1.0, t_amp=0.1, t_k=(np.pi, 2.0, 0.0), t_phase=0.3),
    "density_step": dict(w_density=1.0, target_kind=1, t_lo=0.8, t_hi=1.2, t_n=(1.0, 0.0, 0.0), t_c=0.0),
    "reg": dict(w_reg=10.0, reg_fraction=0.75),
    "all": dict(w_color=1.0, w_grad=0.3, w_density=0.5, w_reg=2.0, reg_fraction=0.75, t_base=1.0, t_amp=0.1,
                t_k=(np.pi, 0.0, 0.0)),
}


@pytest.fixture(scope="module")
def sph():
    from paper_2507_21684_b300 import build
    build.build()
    import paper_2507_21684_b300 as m
    return m


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("term", list(TERMS))
def test_objective_and_gradient_match_oracle(sph, orc, term, walls):
    s = si.shift_problem(16, seed=2, walls=walls)
    loss = TERMS[term]
    with sph.scene_from(s) as sc:
        L, g = sc.shift_gradient(loss)
    nf = s["n_fluid"]
    Lo = orc.shift_objective(s, loss)
    go = orc.shift_gradient(s, loss)
    assert abs(L[0] - Lo) <= 1e-5 * Lo, (L[0], Lo)
    assert rel(g[:nf], go) < 1e-3, rel(g[:nf], go)
    assert np.all(g[nf:] == 0.0)


def test_objective_and_gradient_3d(sph, orc):
    s = si.shift_problem(8, seed=1, dim=3, support=2.5)
    loss = dict(w_color=1.0, w_grad=0.5, w_reg=1.0, reg_fraction=0.6)
    with sph.scene_from(s) as sc:
        L, g = sc.shift_gradient(loss)
    assert abs(L[0] - orc.shift_objective(s, loss)) <= 1e-5 * L[0]
    assert rel(g, orc.shift_gradient(s, loss)) < 1e-3


def test_full_size_directional_derivative(sph, orc):
    """65,536 particles (the paper's backward-cost size): the objective, and the gradient along
    three random directions against the oracle's forward mode."""
    s = si.shift_problem(256, seed=0)
    loss = TERMS["all"]
    with sph.scene_from(s) as sc:
        L, g = sc.shift_gradient(loss)
    Lo = orc.shift_objective(s, loss)
    assert abs(L[0] - Lo) <= 1e-5 * Lo
    rng = np.random.default_rng(3)
    for _ in range(3):
        dirn = rng.standard_normal(g.shape)
        _, dLo = orc.shift_objective(s, loss, None, dirn)
        dL = float((g.astype(np.float64) * dirn).sum())
        assert abs(dL - dLo) <= 1e-3 * np.linalg.norm(g) * np.linalg.norm(dirn), (dL, dLo)


def test_descent_step_and_history(sph, orc):
    s = si.shift_problem(16, seed=4, walls=True)
    loss = dict(w_grad=1.0, w_reg=1.0, reg_fraction=0.5)
    nf = s["n_fluid"]
    go = orc.shift_gradient(s, loss)
    step = float(1e-2 * s["dx"] / np.abs(go).max())
    with sph.scene_from(s) as sc:
        hist = sc.shift_descend(loss, 1, step)
        x1, _, _ = sc.get_state()
    assert abs(hist[0, 0] - orc.shift_objective(s, loss)) <= 1e-5 * hist[0, 0]
    d = x1[:nf].astype(np.float64) - s["x"][:nf]
    assert rel(d, -step * go) < 1e-3
    assert np.array_equal(x1[nf:], s["x"][nf:])  # walls fixed


def test_descent_lowers_the_objective(sph):
    s = si.shift_problem(32, seed=5)
    loss = dict(w_grad=1.0, w_reg=1.0, reg_fraction=0.5)
    with sph.scene_from(s) as sc:
        _, g = sc.shift_gradient(loss)
        step = float(5e-3 * s["dx"] / np.abs(g).max())
        hist = sc.shift_descend(loss, 40, step)
        L_end, _ = sc.shift_gradient(loss)
    h = hist[:, 0]
    assert np.all(np.diff(h) < 0), h
    assert L_end[0] < h[-1] < 0.9 * h[0]
