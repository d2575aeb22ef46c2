"""Oracle pins of the renormalised delta-SPH diffusion (the paper's "Kernel renormalization"
paragraph: L_i = pinv(sum_j V_j (x_j - x_i) (x) grad_i W_ij), corrected gradient
sum_j V_j (A_j - A_i) L_i grad_i W_ij; diffusion term of Antuono et al.).

The renormalised gradient reproduces a linear field exactly wherever M_i has full rank, also
where the support is cut by a free surface; the diffusion built on it vanishes for a linear
density and conserves mass.  Positions and densities are dyadic so that the float32 inputs hold
the linear field exactly."""
import numpy as np
import pytest

from tests.scenes import lattice, params, scene


def _dyadic_block(n_side, dim, seed, jitter_units=40):
    """Lattice of the unit block, dx = 1/n_side (a power of two), jittered by integer multiples
    of 2^-12: every coordinate is exact in float32."""
    dx, x = lattice(n_side, dim)
    rng = np.random.default_rng(seed)
    x = x + rng.integers(-jitter_units, jitter_units + 1, size=x.shape) * 2.0 ** -12
    return dx, x


def _linear_rho(x, b):
    return 1.0 + x @ np.asarray(b, np.float64)


def test_pinv_matches_library_pseudo_inverse(orc):
    """Full rank, rank deficient and indefinite symmetric matrices against numpy's pinv with the
    same relative cut-off (1e-3 of the largest singular value)."""
    rng = np.random.default_rng(0)
    for d in (2, 3):
        for case in range(40):
            Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
            lam = rng.uniform(0.2, 2.0, d)
            if case % 4 == 1:
                lam[0] = 0.0                 # rank deficient
            if case % 4 == 2:
                lam[-1] = -lam[-1]           # indefinite
            if case % 4 == 3:
                lam[0] = 1e-5 * lam.max()    # below the cut-off
            M = (Q * lam) @ Q.T
            L = orc.sym_pinv(M)
            ref = np.linalg.pinv(M, rcond=1e-3, hermitian=True)
            np.testing.assert_allclose(L, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
            if case % 4 == 0:
                np.testing.assert_allclose(L @ M, np.eye(d), atol=1e-12)
            # Moore-Penrose conditions of the retained part
            np.testing.assert_allclose(L @ M @ L, L, atol=1e-10 * max(1.0, np.abs(L).max()))
        assert np.all(orc.sym_pinv(np.zeros((d, d))) == 0.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_renormalised_gradient_exact_for_linear_field_with_free_surface(orc, dim):
    """A block with open faces (no walls, no periodicity): M_i is far from the identity on the
    faces and corners, yet L_i M_i = I makes the gradient of a linear field exact there."""
    n = 32 if dim == 2 else 16
    dx, x = _dyadic_block(n, dim, seed=dim)
    H = 4 * dx if dim == 2 else 2.5 * dx
    p = params(dim=dim, kernel=0 if dim == 2 else 1, H=H, periodic_mask=0, box_lo=(-1,) * dim,
               box_hi=(2,) * dim, diffusion=1)
    b = [0.25, -0.125, 0.0625][:dim]
    rho = _linear_rho(x, b)
    s = scene(p, x, rho=rho, mass=np.full(len(x), dx ** dim))
    assert np.array_equal(s["rho"].astype(np.float64), rho)  # exact in float32
    g, M = orc.renorm_gradient(s, with_M=True)
    np.testing.assert_allclose(g, np.broadcast_to(b, g.shape), rtol=0, atol=1e-10)
    lam = np.linalg.eigvalsh(0.5 * (M + np.transpose(M, (0, 2, 1))))
    assert lam.min() < 0.6       # corners: the support is far from complete
    inner = np.all((x > H * 1.01) & (x < 1 - H * 1.01), axis=1)
    assert np.abs(lam[inner] - 1.0).max() < 0.4    # interior: M_i near the identity (jittered)


def test_renormalisation_matrix_is_identity_on_a_full_periodic_lattice(orc):
    """sum_j V_j (x_j - x_i) (x) grad_i W_ij approximates the integral of (y - x) (x) grad_x W,
    which is the identity; on a regular periodic lattice the sum is symmetric and close to it."""
    dx, x = lattice(32, 2)
    p = params(H=4 * dx, periodic_mask=0b11, diffusion=1)
    s = scene(p, x, mass=np.full(len(x), dx * dx))
    g, M = orc.renorm_gradient(s, with_M=True)
    np.testing.assert_allclose(M, np.broadcast_to(np.eye(2), M.shape), atol=2e-3)
    assert np.all(g == 0.0)  # uniform density


def test_renormalised_diffusion_vanishes_for_a_linear_density(orc):
    """With v = 0 the density rate is the diffusion term alone.  The Molteni-Colagrossi term
    acts on a linear density at the free surface; the renormalised term is zero everywhere."""
    dx, x = _dyadic_block(32, 2, seed=5)
    p0 = params(H=4 * dx, periodic_mask=0, box_lo=(-1, -1), box_hi=(2, 2), nu=0.0, delta=0.1)
    rho = _linear_rho(x, [0.25, -0.125])
    s0 = scene(p0, x, rho=rho, mass=np.full(len(x), dx * dx))
    mc = orc.rates(s0)["drho"]
    s1 = dict(s0, params=dict(p0, diffusion=1))
    rn = orc.rates(s1)["drho"]
    assert np.abs(mc).max() > 1e-3
    assert np.abs(rn).max() < 1e-10 * np.abs(mc).max()


def test_renormalised_diffusion_conserves_mass(orc):
    """psi_ij is symmetric in (i, j) and grad_i W_ij antisymmetric, so sum_i V_i D_i = 0 at any
    state of a periodic box; using only one end's gradient would break it."""
    rng = np.random.default_rng(3)
    dx, x = lattice(24, 2)
    x = (x + rng.uniform(-0.2, 0.2, x.shape) * dx) % 1.0
    p = params(H=4 * dx, periodic_mask=0b11, nu=0.0, delta=0.1, diffusion=1)
    rho = 1.0 + 0.01 * rng.standard_normal(len(x)) + 0.02 * np.sin(2 * np.pi * x[:, 0])
    s = scene(p, x, rho=rho, mass=np.full(len(x), dx * dx))
    d = orc.rates(s)["drho"]
    V = s["mass"].astype(np.float64) / s["rho"].astype(np.float64)
    assert np.abs(d).max() > 0
    assert abs((V * d).sum()) < 1e-13 * np.abs(V * d).sum()
    # and it differs from the Molteni-Colagrossi form on the same state
    d0 = orc.rates(dict(s, params=dict(p, diffusion=0)))["drho"]
    assert np.abs(d - d0).max() > 1e-3 * np.abs(d0).max()


def test_sampled_rates_match_full_rates_in_renormalised_mode(orc):
    """The sampled evaluation gathers the gradients of the sampled particles' neighbours too."""
    import sph_inputs as si
    s = si.taylor_green_2d(32, seed=2, diffusion=1, pressure=True)
    full = orc.rates(s)
    who = np.array([0, 5, 77, 500, 1023], np.int32)
    part = orc.rates(s, who=who)
    np.testing.assert_array_equal(part["drho"], full["drho"][who])
    np.testing.assert_array_equal(part["a"], full["a"][who])


def test_renormalised_mode_has_no_derivative_pass(orc):
    import sph_inputs as si
    s = si.taylor_green_2d(16, seed=0, diffusion=1)
    n, d = s["n_fluid"], 2
    z = np.zeros((n, d))
    with pytest.raises(ValueError):
        orc.adjoint(s, 1, z, z, np.zeros(n))
    with pytest.raises(ValueError):
        orc.jvp(s, 1, s["x"], s["v"], s["rho"], z, z, np.zeros(n))
