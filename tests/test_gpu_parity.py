"""CUDA path vs the FP64 oracle (element by element on seeded inputs).

Bars: cell ranges and neighbour pair sets bit-exact; single-step rates within 1e-5 (normwise
relative, FP32 vs FP64); 10-step rollouts within 1e-3; adjoint gradients within 1e-3 of the
oracle's reverse pass and of central finite differences.
"""
import numpy as np
import pytest

import sph_inputs as si
from tests.scenes import lattice, params, scene

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_max(a, b):
    """Largest elementwise error over the largest reference magnitude: catches a fault confined to
    a few particles (near walls, at periodic edges) that a normwise bound averages away."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)) if b.size else 0.0


@pytest.fixture(scope="module")
def sph():
    from paper_2507_21684_b300 import build
    build.build()
    import paper_2507_21684_b300 as m
    return m


def make(sph, s, **kw):
    return sph.scene_from(s, **kw)


CELL_CASES = {
    "tgv2d_64": lambda: si.taylor_green_2d(64, seed=0),
    "tgv2d_37_ragged": lambda: si.taylor_green_2d(37, seed=3),
    "dambreak_32": lambda: si.dam_break(res=32),
    "tgv3d_20": lambda: si.taylor_green_3d(20, seed=1),
    "tgv2d_16_skin": lambda: si.taylor_green_2d(16, seed=2, skin=0.01, rebuild_interval=4),
    "tgv3d_13_wendland4": lambda: dict(si.taylor_green_3d(13, seed=4),
                                       params=dict(si.taylor_green_3d(13)["params"], kernel=0)),
}


@pytest.mark.parametrize("case", list(CELL_CASES))
def test_cells_bit_exact(sph, orc, case):
    s = CELL_CASES[case]()
    with make(sph, s) as sc:
        start, ids = sc.debug_cells()
    n3, key, oids, ostart = orc.cells(s["params"], s["x"])
    assert np.array_equal(start, ostart)
    assert np.array_equal(ids, oids)


@pytest.mark.parametrize("case", list(CELL_CASES))
def test_pairs_bit_exact(sph, orc, case):
    s = CELL_CASES[case]()
    with make(sph, s) as sc:
        gp = sc.debug_pairs()
    op = orc.pairs(s["params"], s["x"], brute=s["x"].shape[0] <= 3000)
    assert gp.shape == op.shape
    assert np.array_equal(gp, op)


def test_pairs_exact_cutoff_and_periodic_images(sph, orc):
    """d^2 == H^2 is not a neighbour; images across the periodic edge are; unwrapped
    positions several boxes away are folded (floor modulo)."""
    p = params(H=0.25, box_lo=(0, 0), box_hi=(1, 1))
    x = np.array([[0.25, 0.5], [0.5, 0.5],          # exactly H apart: excluded
                  [0.03125, 0.75], [0.96875, 0.75],  # 1/16 apart through the edge
                  [-2.0 + 0.4, 3.0 + 0.1], [0.4, 0.1 + 0.2],  # far unwrapped copy, 0.2 apart
                  [0.7, 0.2]], np.float32)
    s = scene(p, x, mass=np.full(len(x), 1e-3))
    with make(sph, s) as sc:
        gp = sc.debug_pairs()
    op = orc.pairs(p, x, brute=True)
    assert np.array_equal(gp, op)
    assert not any((a, b) == (0, 1) for a, b in gp.tolist())
    assert any((a, b) == (2, 3) for a, b in gp.tolist())


def test_pairs_translation_invariance(sph, orc):
    s = si.taylor_green_2d(24, seed=1)
    x = (np.round(s["x"].astype(np.float64) * 2.0 ** 14) / 2.0 ** 14).astype(np.float32)
    rng = np.random.default_rng(0)
    shift = rng.integers(-3, 4, x.shape).astype(np.float64)
    s0 = dict(s, x=x)
    s1 = dict(s, x=(x + shift).astype(np.float32))
    with make(sph, s0) as a, make(sph, s1) as b:
        pa, pb = a.debug_pairs(), b.debug_pairs()
    assert np.array_equal(pa, pb)
    assert np.array_equal(pa, orc.pairs(s["params"], x, brute=True))


@pytest.mark.parametrize("n", [1, 2, 31, 33])
def test_tiny_and_ragged_counts(sph, orc, n):
    s = si.taylor_green_2d(16, seed=5)
    sub = dict(s, x=s["x"][:n].copy(), v=s["v"][:n].copy(), rho=s["rho"][:n].copy(), mass=s["mass"][:n].copy(),
               n_fluid=n)
    with make(sph, sub) as sc:
        gp = sc.debug_pairs()
        r = sc.rates()
        sc.step(3)
        x, v, rho = sc.get_state()
    assert np.array_equal(gp, orc.pairs(s["params"], sub["x"], brute=True))
    o = orc.rates(sub)
    assert rel(r["a"], o["a"]) < 1e-5
    xo, vo, ro = orc.rollout(sub, 3)
    assert rel(x - sub["x"], xo - sub["x"]) < 1e-4


def _snapshot(orc, s, steps):
    """Oracle state after `steps` steps, rounded to float32 (so both sides see the same input)."""
    xo, vo, ro = orc.rollout(s, steps)
    return dict(s, x=xo.astype(np.float32), v=vo.astype(np.float32), rho=ro.astype(np.float32))


def _summation(s):
    return dict(s, params=dict(s["params"], density_mode=1))


RATE_CASES = {
    "tgv2d_64_t0": lambda orc: si.taylor_green_2d(64, seed=0),
    "tgv2d_64_pressure_t0": lambda orc: si.taylor_green_2d(64, seed=6, pressure=True),
    "tgv2d_64_t20": lambda orc: _snapshot(orc, si.taylor_green_2d(64, seed=0), 20),
    "dambreak_64_t20": lambda orc: _snapshot(orc, si.dam_break(res=64), 20),
    "tgv3d_24_t10": lambda orc: _snapshot(orc, si.taylor_green_3d(24, seed=2), 10),
    "tgv2d_48_summation_t10": lambda orc: _snapshot(orc, si.taylor_green_2d(48, seed=1, density_mode=1), 10),
    "dambreak_48_summation_t10": lambda orc: _snapshot(orc, _summation(si.dam_break(res=48)), 10),
}


@pytest.mark.parametrize("case", list(RATE_CASES))
def test_single_step_rates(sph, orc, case):
    s = RATE_CASES[case](orc)
    with make(sph, s) as sc:
        g = sc.rates()
    o = orc.rates(s)
    ea, ed = rel(g["a"], o["a"]), rel(g["drho"], o["drho"])
    er = rel(g["rho"], o["rho"])
    assert ea < 1e-5, ea
    if s["params"]["density_mode"] == 0:
        assert ed < 1e-5, ed
    assert er < 1e-6, er
    # elementwise: no particle's rate off by more than 1e-4 of the field's largest value
    ma, md = rel_max(g["a"], o["a"]), rel_max(g["drho"], o["drho"])
    assert ma < 1e-4, ma
    if s["params"]["density_mode"] == 0:
        assert md < 1e-4, md


ROLL_CASES = {
    "tgv2d_64": lambda: si.taylor_green_2d(64, seed=0),
    "dambreak_128_full": lambda: si.dam_break(res=128),
    "tgv3d_32": lambda: si.taylor_green_3d(32, seed=1),
    "tgv2d_32_summation": lambda: si.taylor_green_2d(32, seed=2, density_mode=1),
    "dambreak_64_summation": lambda: _summation(si.dam_break(res=64)),
    # 3D in summation mode with a Verlet skin: the density pass and the warp-per-tile sweep on cells
    # rebuilt in conditional graph nodes, with x sub-bins
    "tgv3d_20_summation_skin": lambda: _verlet(_summation(si.taylor_green_3d(20, seed=6)), 0.1),
    "tgv2d_32_verlet": lambda: si.taylor_green_2d(32, seed=2, skin=0.02, rebuild_interval=5),
}


def quant_floor(ref):
    """Norm of half an ulp of the float32 output at the reference values: the part of any
    float32 result's error that no arithmetic can remove."""
    r = np.asarray(ref, np.float64)
    return float(np.linalg.norm(0.5 * np.spacing(np.abs(r).astype(np.float32)).astype(np.float64)))


def check_rollout(s, n, x, v, rho, xo, vo, ro, tol=1e-3):
    """Normwise relative errors of displacement, velocity and density change; each bound is
    tol * |reference| plus the float32 output quantisation of that field."""
    x0 = s["x"].astype(np.float64)
    r0 = s["params"]["rho0"]
    dx_err = np.linalg.norm((x - x0) - (xo - x0))
    assert dx_err <= tol * np.linalg.norm(xo - x0) + quant_floor(xo), (dx_err, np.linalg.norm(xo - x0))
    assert np.linalg.norm(v - vo) <= tol * np.linalg.norm(vo) + quant_floor(vo)
    assert np.linalg.norm((rho - r0) - (ro - r0)) <= tol * np.linalg.norm(ro - r0) + quant_floor(ro)


@pytest.mark.parametrize("case", list(ROLL_CASES))
def test_ten_step_rollout(sph, orc, case):
    s = ROLL_CASES[case]()
    n = 10
    with make(sph, s) as sc:
        sc.step(n)
        x, v, rho = sc.get_state()
    xo, vo, ro = orc.rollout(s, n)
    check_rollout(s, n, x, v, rho, xo, vo, ro)


def test_dam_break_hundred_steps(sph, orc):
    """100 steps of the full dam break: the displacement now dwarfs the float32 spacing."""
    s = si.dam_break(res=128)
    with make(sph, s) as sc:
        sc.step(100)
        x, v, rho = sc.get_state()
    xo, vo, ro = orc.rollout(s, 100)
    x0 = s["x"].astype(np.float64)
    assert rel(x - x0, xo - x0) < 1e-3
    assert rel(v, vo) < 1e-3
    assert rel(rho - 1.0, ro - 1.0) < 1e-3


def _verlet(s, skin_over_H, interval=1 << 20):
    p = dict(s["params"])
    p["skin"] = float(np.float32(skin_over_H * p["H"]))
    p["rebuild_interval"] = int(interval)
    return dict(s, params=p)


@pytest.mark.parametrize("case,skin,n", [("tgv2d_64", 0.1, 40), ("dambreak_128", 0.02, 300), ("tgv3d_24", 0.1, 40)])
def test_verlet_skin_rebuilds_on_displacement(sph, orc, case, skin, n):
    """Skin and no interval limit: the device-side displacement check alone decides when the cells
    are rebuilt (fewer rebuilds than steps, more than the initial one), and the rollout still
    matches the oracle, which searches neighbours every step.  In 3D the rebuilds order the cells
    by x sub-bin for the warp-per-tile sweep."""
    base = {"tgv2d_64": lambda: si.taylor_green_2d(64, seed=0), "dambreak_128": lambda: si.dam_break(res=128),
            "tgv3d_24": lambda: si.taylor_green_3d(24, seed=3)}[case]()
    s = _verlet(base, skin)
    with make(sph, s) as sc:
        sc.step(n)
        st = sc.stats()
        x, v, rho = sc.get_state()
    assert st["steps"] == n
    assert 1 < st["rebuilds"] < n, st
    xo, vo, ro = orc.rollout(s, n)
    x0 = s["x"].astype(np.float64)
    assert rel(x - x0, xo - x0) < 1e-3
    assert rel(v, vo) < 1e-3
    r0 = s["params"]["rho0"]
    assert rel(rho - r0, ro - r0) < 1e-3


def test_verlet_interval_counts_rebuilds_and_launches(sph):
    """Skin wide enough that displacement never triggers: cells serve exactly `interval` sweeps
    (the initial host build, then a conditional rebuild every 3rd step), and the launch counter
    includes the kernels of the rebuilds taken inside the graphs."""
    s = _verlet(si.taylor_green_2d(32, seed=1), 0.5, interval=3)
    with make(sph, s) as sc:
        sc.step(30)
        st = sc.stats()
        _, launches = sc.counters()
        sc.step(30)
        st2 = sc.stats()
        _, launches2 = sc.counters()
    assert st["rebuilds"] == 10, st
    assert st2["rebuilds"] - st["rebuilds"] == 10, st2  # steps 31..60: rebuilds at 31, 34, ..., 58
    assert launches2 >= 2 * 30  # at least the decision and the sweep of every step
    assert st2["launches"] - st["launches"] == launches2


def test_graph_replay_is_bitwise_eager(sph):
    s = si.taylor_green_2d(48, seed=3)
    with make(sph, s) as a, make(sph, s) as b:
        a.step(24)  # graph chunks
        for _ in range(24):
            b.step(1)  # eager
        xa, va, ra = a.get_state()
        xb, vb, rb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(ra, rb)


def test_rollout_equals_step(sph):
    s = si.taylor_green_2d(32, seed=3)
    with make(sph, s) as a, make(sph, s) as b:
        a.step(30)
        b.rollout(30, 7)
        assert all(np.array_equal(p, q) for p, q in zip(a.get_state(), b.get_state()))


def test_adjoint_matches_oracle_and_fd(sph, orc):
    """Config of the adjoint workload on the 16 x 16 copy: 200 steps, checkpoints every 20,
    loss = mean squared final-position error against a target rollout from perturbed v0."""
    s = si.adjoint_problem(16)
    steps, vt = 200, s["v_target"]
    N = s["n_fluid"]
    xt, _, _ = orc.rollout(s, steps, v=vt)
    with make(sph, s) as sc:
        sc.rollout(steps, 20)
        xT, vT, rT = sc.get_state()
        seed = (2.0 * (xT.astype(np.float64) - xt) / N).astype(np.float32)
        gx, gv, gr, gnu = sc.adjoint(seed, np.zeros_like(seed), np.zeros(N, np.float32))
    x0, v0, r0 = (s[k].astype(np.float64) for k in ("x", "v", "rho"))
    xo, _, _ = orc.rollout64(s, steps, x0, v0, r0)
    oseed = 2.0 * (xo - xt) / N
    o = orc.adjoint(s, steps, oseed, np.zeros_like(oseed), np.zeros(N), x=x0, v=v0, rho=r0)
    assert rel(gv, o["vb"]) < 1e-3
    assert rel(gx, o["xb"]) < 1e-3
    assert abs(gnu - o["nub"]) < 1e-3 * abs(o["nub"])

    def loss(v, nu=None):
        xx, _, _ = orc.rollout64(s, steps, x0, v, r0, nu=nu)
        return ((xx - xt) ** 2).sum() / N

    rng = np.random.default_rng(7)
    for _ in range(3):
        dv = rng.standard_normal(v0.shape)
        h = 1e-6
        fd = (loss(v0 + h * dv) - loss(v0 - h * dv)) / (2 * h)
        assert abs((gv.astype(np.float64) * dv).sum() - fd) < 1e-3 * abs(fd)
    nu = s["params"]["nu"]
    h = 1e-7
    fd_nu = (loss(v0, nu + h) - loss(v0, nu - h)) / (2 * h)
    assert abs(gnu - fd_nu) < 1e-3 * abs(fd_nu)


def _adjoint_vs_oracle(sph, orc, s, steps=200, replay=0):
    vt = s["v_target"]
    N = s["n_fluid"]
    xt, _, _ = orc.rollout(s, steps, v=vt)
    with make(sph, s) as sc:
        sc.set_adjoint_replay(replay)
        sc.rollout(steps, 20)
        xT, _, _ = sc.get_state()
        seed = (2.0 * (xT.astype(np.float64) - xt) / N).astype(np.float32)
        gx, gv, gr, gnu = sc.adjoint(seed, None, None)
        info = sc.adjoint_info()
    x0, v0, r0 = (s[k].astype(np.float64) for k in ("x", "v", "rho"))
    xo, _, _ = orc.rollout64(s, steps, x0, v0, r0)
    oseed = 2.0 * (xo - xt) / N
    o = orc.adjoint(s, steps, oseed, np.zeros_like(oseed), np.zeros(N), x=x0, v=v0, rho=r0)
    return gx, gv, gnu, o, info


@pytest.mark.parametrize("skin_over_H,replay,expect_fallback", [(0.3, 0, False), (0.002, 16, True)])
def test_adjoint_replay_on_a_skin(sph, orc, skin_over_H, replay, expect_fallback):
    """With a Verlet skin the adjoint's forward replay rebuilds every few steps (from the
    rollout's rebuild rate); a skin too thin for a forced interval of 16 makes the replay fall back
    to a rebuild every step.  Either way the gradients are the oracle's."""
    s = si.adjoint_problem(16)
    p = dict(s["params"], skin=float(np.float32(skin_over_H * s["params"]["H"])), rebuild_interval=1 << 20)
    s = dict(s, params=p)
    gx, gv, gnu, o, info = _adjoint_vs_oracle(sph, orc, s, replay=replay)
    assert rel(gv, o["vb"]) < 1e-3
    assert rel(gx, o["xb"]) < 1e-3
    assert abs(gnu - o["nub"]) < 1e-3 * abs(o["nub"])
    assert (info["replay_fallbacks"] > 0) == expect_fallback, info
    if not expect_fallback:
        assert info["replay_interval"] > 1


def test_autograd_function_matches_adjoint(sph):
    """rollout_fn (torch.autograd.Function: forward sph_rollout, backward sph_adjoint) gives the
    gradients of the direct adjoint call, for a loss on the final positions."""
    import torch
    s = si.adjoint_problem(16, steps=40)
    N = s["n_fluid"]
    tgt = torch.from_numpy(s["x"]).cuda() + 0.01
    f = sph.rollout_fn()
    x0 = torch.from_numpy(s["x"]).cuda()
    v0 = torch.from_numpy(s["v"]).cuda().requires_grad_(True)
    r0 = torch.from_numpy(s["rho"]).cuda()
    nu = torch.tensor(s["params"]["nu"], device="cuda", requires_grad=True)
    m = torch.from_numpy(s["mass"]).cuda()
    xT, vT, rT = f.apply(x0, v0, r0, nu, m, s["params"], 40, 10)
    loss = ((xT - tgt) ** 2).sum() / N
    loss.backward()
    with make(sph, s) as sc:
        sc.rollout(40, 10)
        x, _, _ = sc.get_state()
        seed = (2.0 * (x.astype(np.float64) - tgt.cpu().numpy()) / N).astype(np.float32)
        gx, gv, gr, gnu = sc.adjoint(seed, np.zeros_like(seed), np.zeros(N, np.float32))
    np.testing.assert_allclose(v0.grad.cpu().numpy(), gv, rtol=1e-5, atol=1e-9)
    assert abs(float(nu.grad) - gnu) <= 1e-5 * abs(gnu)


def test_checkpoint_recompute_is_bitwise_store_all(sph):
    s = si.taylor_green_2d(16, seed=1)
    N = s["n_fluid"]
    rng = np.random.default_rng(1)
    seed = rng.standard_normal((N, 2)).astype(np.float32)
    out = []
    for k in (5, 40):
        with make(sph, s) as sc:
            sc.rollout(40, k)
            out.append(sc.adjoint(seed, seed, np.ones(N, np.float32)))
    for a, b in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(a, b)
    assert out[0][3] == out[1][3]


def test_adjoint_full_size_matches_oracle(sph, orc):
    """128 x 128 copy of the adjoint workload, 200 steps, checkpoints every 20."""
    s = si.adjoint_problem(128)
    steps, vt = 200, s["v_target"]
    N = s["n_fluid"]
    xt, _, _ = orc.rollout(s, steps, v=vt)
    with make(sph, s) as sc:
        sc.rollout(steps, 20)
        xT, _, _ = sc.get_state()
        seed = (2.0 * (xT.astype(np.float64) - xt) / N).astype(np.float32)
        gx, gv, gr, gnu = sc.adjoint(seed, None, None)
    x0, v0, r0 = (s[k].astype(np.float64) for k in ("x", "v", "rho"))
    xo, _, _ = orc.rollout64(s, steps, x0, v0, r0)
    o = orc.adjoint(s, steps, 2.0 * (xo - xt) / N, np.zeros_like(xo), np.zeros(N), x=x0, v=v0, rho=r0)
    assert rel(gv, o["vb"]) < 1e-3
    assert abs(gnu - o["nub"]) < 1e-3 * abs(o["nub"])


def test_full_size_3d_rates_sampled(sph, orc):
    """2,097,152-particle 3D Taylor-Green (Wendland C2) with its analytic pressure field:
    rates of 4096 sampled particles against the oracle, same launch path as the benchmark."""
    s = si.taylor_green_3d(128, seed=0, pressure=True)
    with make(sph, s) as sc:
        g = sc.rates()
    idx = np.arange(0, s["n_fluid"], 512, dtype=np.int32)
    o = orc.rates(s, who=idx)
    assert rel(g["a"][idx], o["a"]) < 1e-5
    assert rel(g["drho"][idx], o["drho"]) < 1e-5


def test_full_size_3d_headline_steps(sph, orc):
    """The benchmark's launch configuration: 2,097,152-particle 3D Taylor-Green with the tuned
    Verlet skin of 0.05 H, graph-launched steps (the warp-per-tile sweep in CTAs of 24 warps, x
    sub-bins, device-decided rebuilds in conditional graph nodes); five steps against the FP64
    oracle's rollout over every particle."""
    s = _verlet(si.taylor_green_3d(128, seed=0), 0.05)
    n = 5
    with make(sph, s) as sc:
        sc.step(n)
        st = sc.stats()
        x, v, rho = sc.get_state()
    assert 1 <= st["rebuilds"] <= n, st
    xo, vo, ro = orc.rollout(s, n)
    check_rollout(s, n, x, v, rho, xo, vo, ro)


def test_3d_closed_box_with_walls_rollout(sph, orc):
    """3D scene in a closed box (no periodic axis) with three layers of wall particles around the
    fluid: the warp-per-tile sweep's clamped windows at the box faces, the 3D wall pass (Shepard
    extrapolation with gravity) and the fluid's rollout against the oracle."""
    s = si.shift_problem(12, seed=5, dim=3, walls=True)
    n, nf = len(s["x"]), s["n_fluid"]
    rng = np.random.default_rng(3)
    v = np.zeros((n, 3), np.float32)
    v[:nf] = (0.3 * rng.standard_normal((nf, 3))).astype(np.float32)
    p = dict(s["params"], nu=0.01, delta=0.1, g=[0.0, 0.0, -1.0])
    s = dict(s, v=v, params=p)
    nsteps = 10
    with make(sph, s) as sc:
        sc.step(nsteps)
        x, v1, rho = sc.get_state()
    xo, vo, ro = orc.rollout(s, nsteps)
    check_rollout(dict(s, x=s["x"][:nf]), nsteps, x[:nf], v1[:nf], rho[:nf], xo[:nf], vo[:nf], ro[:nf])


def test_instability_is_reported(sph):
    s = si.taylor_green_2d(16, seed=0)
    s = dict(s, v=(s["v"] * 200.0).astype(np.float32))
    with make(sph, s) as sc:
        sc.step(20)
        with pytest.raises(sph.SphError) as e:
            sc.get_state()
        assert e.value.code == sph.SPH_EUNSTABLE


def test_device_inputs_match_host_inputs(sph):
    import torch
    s = si.taylor_green_2d(32, seed=4)
    with make(sph, s) as a, make(sph, s, device=True) as b:
        a.step(5)
        b.step(5)
        xa, va, ra = a.get_state()
        xb, vb, rb = b.get_state(device=True)
        torch.cuda.synchronize()
    assert np.array_equal(xa, xb.cpu().numpy()) and np.array_equal(va, vb.cpu().numpy())


def _sparse_line_scene():
    """Clusters of two particles every three cells along one cell line: cut at whole cells, a tile
    of 64 particles would span more cells than the staged column table holds (global-memory
    fallback path); cut into balanced tiles, the chunks of TP cells bound the span."""
    H = 0.01
    p = params(H=H, dt=1e-4, box_lo=(0, 0), box_hi=(4, 0.1), periodic_mask=0b01, nu=0.01)
    xs = []
    for c in range(120):
        x0 = (3 * c + 0.5) * H
        xs += [[x0, 0.05], [x0 + 0.4 * H, 0.05 + 0.3 * H]]
    x = np.array(xs)
    rng = np.random.default_rng(0)
    v = rng.standard_normal(x.shape) * 0.1
    rho = 1.0 + 0.01 * rng.standard_normal(len(x))
    return scene(p, x, v=v, rho=rho, mass=np.full(len(x), H * H / 16))


def _clump_scene():
    """A dense clump (1500 particles inside one cell) next to a sparse lattice: the staged region
    exceeds shared memory (global-memory fallback path)."""
    p = params(H=0.1, dt=1e-4, box_lo=(0, 0), box_hi=(1, 1), periodic_mask=0b11, nu=0.01)
    rng = np.random.default_rng(1)
    clump = 0.45 + 0.09 * rng.random((1500, 2))
    dx, lat = lattice(32, 2)
    x = np.concatenate([clump, lat])
    rho = 1.0 + 0.01 * rng.standard_normal(len(x))
    return scene(p, x, v=0.1 * rng.standard_normal(x.shape), rho=rho, mass=np.full(len(x), 1e-4))


def _long_line_scene():
    """Cell lines of 2500 cells (more than 32 chunks of TP cells: the balanced tiler's second
    window), with a lattice strip, clusters straddling the chunk boundaries (multiples of 32 and
    64 cells), an over-full cell of 150 particles and scattered particles."""
    H = 0.01
    p = params(H=H, dt=1e-4, box_lo=(0, 0), box_hi=(25, 0.05), periodic_mask=0b11, nu=0.01)
    rng = np.random.default_rng(7)
    parts = [np.stack([rng.uniform(0, 25, 1200), rng.uniform(0, 0.05, 1200)], 1)]
    gx, gy = np.meshgrid(np.arange(0.0, 1.2, 0.25 * H), np.arange(0.0, 0.05, 0.25 * H))
    parts.append(np.stack([gx.ravel() + 20.0, gy.ravel()], 1))
    for c in (32, 64, 96, 128, 1024, 2048, 2080):
        parts.append(np.stack([c * H + rng.uniform(-1.5 * H, 1.5 * H, 40), rng.uniform(0, 0.05, 40)], 1))
    parts.append(np.stack([13.0 + rng.uniform(0, 0.9 * H, 150), 0.02 + rng.uniform(0, 0.9 * H, 150)], 1))
    x = np.concatenate(parts)
    v = rng.standard_normal(x.shape) * 0.1
    rho = 1.0 + 0.01 * rng.standard_normal(len(x))
    return scene(p, x, v=v, rho=rho, mass=np.full(len(x), H * H / 16))


@pytest.mark.parametrize("maker", [_sparse_line_scene, _clump_scene, _long_line_scene])
def test_fallback_tiles_match_oracle(sph, orc, maker):
    s = maker()
    with make(sph, s) as sc:
        g = sc.rates()
        gp = sc.debug_pairs()
    o = orc.rates(s)
    assert rel(g["a"], o["a"]) < 1e-5
    assert rel(g["drho"], o["drho"]) < 1e-5
    assert np.array_equal(gp, orc.pairs(s["params"], s["x"], brute=True))


def _batch_specs():
    a = si.taylor_green_2d(16, seed=1)
    b = si.taylor_green_2d(40, seed=2, nu=0.02)
    c = si.taylor_green_2d(24, seed=3, pressure=True)
    return [a, b, c]


@pytest.mark.parametrize("skin", [0.0, 0.02])
def test_batched_wall_scenes_bitwise_equal_alone(sph, skin):
    """Dam breaks of different sizes with a periodic scene in one batch: the fused wall + sweep
    launch (wall tasks of every scene first) gives each scene the bits it gets alone when every step
    rebuilds; with a skin the batch rebuilds whenever any scene needs it, so the sums may run in
    another order: equal to float rounding."""
    raw = [si.dam_break(res=32), si.taylor_green_2d(24, seed=3), si.dam_break(res=48)]
    absolute = float(np.float32(skin * min(s["params"]["H"] for s in raw)))  # one skin for the batch

    def sk(s):
        p = dict(s["params"], skin=absolute, rebuild_interval=1 if skin == 0 else 1 << 20)
        return dict(s, params=p)
    specs = [sk(s) for s in raw]
    with sph.Scene.batch(specs) as bt:
        bt.step(17)
        xb, vb, rb = bt.get_state()
        rows = list(zip(bt.first_row, bt.rows))
    for spec, (f, n) in zip(specs, rows):
        with make(sph, spec) as sc:
            sc.step(17)
            x, v, r = sc.get_state()
        if skin == 0.0:
            assert np.array_equal(x, xb[f:f + n]) and np.array_equal(v, vb[f:f + n]) and np.array_equal(r, rb[f:f + n])
        else:
            x0 = spec["x"].astype(np.float64)
            assert rel(xb[f:f + n] - x0, x - x0) < 1e-4
            assert rel(vb[f:f + n], v) < 1e-4
            assert rel(rb[f:f + n] - 1.0, r - 1.0) < 1e-4


def test_batched_scenes_bitwise_equal_alone(sph):
    """Packing scenes into one batch (shared launches) changes no bit of any scene's result."""
    specs = _batch_specs()
    with sph.Scene.batch(specs) as bt:
        bt.step(13)
        xb, vb, rb = bt.get_state()
        rows = list(zip(bt.first_row, bt.rows))
    for spec, (f, n) in zip(specs, rows):
        with make(sph, spec) as sc:
            sc.step(13)
            x, v, r = sc.get_state()
        assert np.array_equal(x, xb[f:f + n]) and np.array_equal(v, vb[f:f + n]) and np.array_equal(r, rb[f:f + n])


def test_batched_3d_scenes_bitwise_equal_alone(sph, orc):
    """3D scenes of different sizes and parameters in one batch, swept by the warp-per-tile
    traversal (tiles of several scenes in one launch): every scene's result is the bits it gets
    alone, and the first matches the oracle's 5-step rollout."""
    specs = [si.taylor_green_3d(10, seed=1), si.taylor_green_3d(14, seed=2, nu=0.01),
             si.taylor_green_3d(12, seed=3, pressure=True)]
    with sph.Scene.batch(specs) as bt:
        bt.step(5)
        xb, vb, rb = bt.get_state()
        rows = list(zip(bt.first_row, bt.rows))
    for spec, (f, n) in zip(specs, rows):
        with make(sph, spec) as sc:
            sc.step(5)
            x, v, r = sc.get_state()
        assert np.array_equal(x, xb[f:f + n]) and np.array_equal(v, vb[f:f + n]) and np.array_equal(r, rb[f:f + n])
    xo, vo, ro = orc.rollout(specs[0], 5)
    f, n = rows[0]
    check_rollout(specs[0], 5, xb[f:f + n], vb[f:f + n], rb[f:f + n], xo, vo, ro)


def test_batched_3d_scenes_with_a_skin_match_alone_and_oracle(sph, orc):
    """3D scenes with Verlet skins in one batch (cells rebuilt in conditional graph nodes with x
    sub-bins, the whole batch whenever one scene needs it): each scene equals its result alone to
    float rounding (its sums may run in another order), and the first matches the oracle."""
    raw = [si.taylor_green_3d(12, seed=1), si.taylor_green_3d(16, seed=2, nu=0.01), si.taylor_green_3d(10, seed=4)]
    specs = [_verlet(s, 0.1) for s in raw]
    n = 12
    with sph.Scene.batch(specs) as bt:
        bt.step(n)
        st = bt.stats()
        xb, vb, rb = bt.get_state()
        rows = list(zip(bt.first_row, bt.rows))
    assert 1 <= st["rebuilds"] < n, st
    for spec, (f, m) in zip(specs, rows):
        with make(sph, spec) as sc:
            sc.step(n)
            x, v, r = sc.get_state()
        x0 = spec["x"].astype(np.float64)
        assert rel(xb[f:f + m] - x0, x - x0) < 1e-4
        assert rel(vb[f:f + m], v) < 1e-4
        assert rel(rb[f:f + m] - 1.0, r - 1.0) < 1e-4
    xo, vo, ro = orc.rollout(specs[0], n)
    f, m = rows[0]
    check_rollout(specs[0], n, xb[f:f + m], vb[f:f + m], rb[f:f + m], xo, vo, ro)


def test_batched_adjoint_bitwise_equal_alone(sph):
    specs = _batch_specs()
    rng = np.random.default_rng(3)
    seeds = [rng.standard_normal((s["n_fluid"], 2)).astype(np.float32) for s in specs]
    with sph.Scene.batch(specs) as bt:
        bt.rollout(30, 10)
        gx, gv, gr, gnu = bt.adjoint(np.concatenate(seeds), None, None)
        rows = list(zip(bt.first_row, bt.rows))
    for spec, sd, (f, n), nu_b in zip(specs, seeds, rows, gnu):
        with make(sph, spec) as sc:
            sc.rollout(30, 10)
            ax, av, ar, anu = sc.adjoint(sd, None, None)
        assert np.array_equal(ax, gx[f:f + n]) and np.array_equal(av, gv[f:f + n])
        assert anu == nu_b


def test_bounded_device_waits_give_up_and_the_context_survives(sph):
    """The fused kernel's gate wait and the cooperative rebuild's grid barrier are bounded: made to
    wait for something that never happens (no fault), each gives up, reports status bit 1, and
    the next scene runs normally."""
    import ctypes as C
    import time
    g, b = C.c_int(0), C.c_int(0)
    t0 = time.perf_counter()
    rc = sph.lib().sph_debug_bounded_waits(C.byref(g), C.byref(b))
    dt = time.perf_counter() - t0
    assert rc == sph.SPH_OK
    assert g.value & 2 and b.value & 2
    assert dt < 30.0
    s = si.taylor_green_2d(16, seed=0)
    with make(sph, s) as sc:
        sc.step(3)
        x, _, _ = sc.get_state()
    assert np.all(np.isfinite(x))
