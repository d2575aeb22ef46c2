"""Oracle pins of the variable support radius (the paper's symmetric neighbour search for
per-particle radii): pair set under max(h_i, h_j), the search radius s_i, super-symmetric and
gather densities."""
import numpy as np
import pytest

import sph_inputs as si
from tests.scenes import lattice, params, scene


def _radii(n, H, seed, lo=0.55):
    rng = np.random.default_rng(seed)
    return (H * rng.uniform(lo, 1.0, n)).astype(np.float32)


def test_uniform_radii_reduce_to_the_plain_scheme(orc):
    s = si.taylor_green_2d(24, seed=1)
    p = s["params"]
    h = np.full(s["n_fluid"], p["H"], np.float32)
    out = orc.support(s, h)
    assert np.all(out["search_radius"] == p["H"])
    rho = orc.rates(dict(s, params=dict(p, density_mode=1)))["rho"]
    np.testing.assert_allclose(out["rho_super"], rho, rtol=1e-13)
    np.testing.assert_allclose(out["rho_gather"], rho, rtol=1e-13)
    assert np.array_equal(orc.pairs_var(s, h), orc.pairs(p, s["x"], brute=True))


def test_search_radius_covers_every_pair_and_is_a_given_radius(orc):
    s = si.taylor_green_2d(20, seed=3)
    p = s["params"]
    h = _radii(s["n_fluid"], p["H"], 5)
    prs = orc.pairs_var(s, h)
    out = orc.support(s, h)
    sr = out["search_radius"]
    # symmetric pair set
    fwd = set(map(tuple, prs))
    assert all((j, i) in fwd for i, j in fwd)
    # every pair lies within the search radius of both ends
    x = s["x"].astype(np.float64)
    r = x[prs[:, 0]] - x[prs[:, 1]]
    r -= np.round(r)  # unit periodic box
    d = np.sqrt((r ** 2).sum(1))
    assert np.all(d < sr[prs[:, 0]]) and np.all(d < sr[prs[:, 1]])
    # s_i is h_i or the radius of a particle whose support holds i
    hd = h.astype(np.float64)
    for i in range(0, s["n_fluid"], 7):
        cands = {hd[i]} | {hd[j] for a, j in prs if a == i and d[(prs[:, 0] == i) & (prs[:, 1] == j)][0] < hd[j]}
        assert sr[i] == max(cands)
    # the pairs with different radii include some that only the larger radius admits
    hm = np.maximum(hd[prs[:, 0]], hd[prs[:, 1]])
    hn = np.minimum(hd[prs[:, 0]], hd[prs[:, 1]])
    assert np.any(d >= hn) and np.all(d < hm)


def test_two_particles_closed_form(orc):
    """A (h = H) and B (h = H/2) at distance 0.75 H: they interact (max rule), B's search radius
    grows to H, B's gather density sees only itself, its super-symmetric density half of A's
    kernel."""
    H = 0.25
    p = params(H=H, periodic_mask=0, box_lo=(-1, -1), box_hi=(2, 2))
    x = np.array([[0.5, 0.5], [0.5 + 0.75 * H, 0.5]])
    s = scene(p, x, mass=np.array([1.0, 2.0]))
    h = np.array([H, H / 2], np.float32)
    out = orc.support(s, h)
    assert out["search_radius"][1] == H and out["search_radius"][0] == H
    assert orc.pairs_var(s, h).tolist() == [[0, 1], [1, 0]]
    W = lambda r, hh: orc.kernel_eval(dict(p, H=float(hh)), [r, 0.0])[0]
    assert out["rho_gather"][1] == pytest.approx(2.0 * W(0.0, H / 2), rel=1e-14)
    assert out["rho_super"][1] == pytest.approx(2.0 * W(0.0, H / 2) + 1.0 * 0.5 * W(0.75 * H, H), rel=1e-14)
    assert out["rho_gather"][0] == pytest.approx(1.0 * W(0.0, H) + 2.0 * W(0.75 * H, H), rel=1e-14)


def test_gather_density_is_normalised_for_any_radius(orc):
    """On a regular lattice the gather density with any radius h_i of a few spacings is the
    lattice density m / dx^2 to the kernel's discretisation error (integral of W = 1)."""
    dx, x = lattice(32, 2)
    p = params(H=4 * dx, periodic_mask=0b11)
    s = scene(p, x, mass=np.full(len(x), dx * dx))
    h = _radii(len(x), p["H"], 2, lo=0.7)
    out = orc.support(s, h)
    np.testing.assert_allclose(out["rho_gather"], 1.0, atol=2e-2)
