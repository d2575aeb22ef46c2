"""Serving loop: continuous batching gives each request the same result as running it alone;
admission honours the HBM budget; waits are bounded."""
import time

import numpy as np
import pytest

import sph_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    from paper_2507_21684_b300 import build
    build.build()
    import paper_2507_21684_b300 as m
    return m


def _alone(sph, spec, steps, adjoint=False, ckpt=20, x_target=None):
    with sph.scene_from(spec) as sc:
        if not adjoint:
            sc.step(steps)
            return dict(zip(("x", "v", "rho"), sc.get_state()))
        sc.rollout(steps, ckpt)
        x, v, r = sc.get_state()
        tgt = spec["x"] if x_target is None else x_target
        seed = (2.0 * (x.astype(np.float64) - tgt) / spec["n_fluid"]).astype(np.float32)
        gx, gv, gr, nub = sc.adjoint(seed, None, None)
        return dict(x=x, v=v, rho=r, xbar0=gx, vbar0=gv, rhobar0=gr, nubar=nub)


def test_served_results_equal_alone(sph):
    specs = [si.taylor_green_2d(n, seed=k) for k, n in enumerate([16, 40, 24, 32, 20])]
    steps = [13, 31, 7, 20, 26]
    adj = [False, False, True, False, True]
    with sph.Server(8 << 30, 64) as sv:
        tickets = []
        for sp, st, a in zip(specs, steps, adj):
            tickets.append(sv.submit(sp, st, adjoint=a, ckpt_every=5))
            time.sleep(0.002)  # staggered arrivals: requests join a batch that is already running
        got = [sv.wait(t) for t in tickets]
        info = sv.stats()
    assert info["repacks"] >= 2
    for sp, st, a, g in zip(specs, steps, adj, got):
        ref = _alone(sph, sp, st, adjoint=a, ckpt=5)
        for k in ("x", "v", "rho"):
            assert np.array_equal(g[k], ref[k]), k
        if a:
            for k in ("xbar0", "vbar0", "rhobar0"):
                assert np.array_equal(g[k], ref[k]), k
            assert g["nubar"] == ref["nubar"]


def test_served_with_a_skin_and_summation_adjoints_match_alone(sph):
    """Requests with a Verlet skin (a batch rebuilds all its scenes when one needs it, so a scene
    may be re-sorted on other steps than alone: the same neighbours summed in another order) equal
    their results alone to rounding; adjoint requests in summation mode, on the adjoint workers,
    equal theirs bitwise."""
    def skinned(sp):
        p = dict(sp["params"], skin=float(np.float32(0.1 * sp["params"]["H"])), rebuild_interval=1 << 20)
        return dict(sp, params=p)
    specs = [skinned(si.taylor_green_2d(n, seed=k)) for k, n in enumerate([16, 40, 24, 32])]
    steps = [40, 61, 27, 50]
    adj_specs = [si.taylor_green_2d(n, seed=10 + k, density_mode=1) for k, n in enumerate([16, 20, 24])]
    with sph.Server(8 << 30, 64) as sv:
        tickets = []
        for sp, st in zip(specs, steps):
            tickets.append(sv.submit(sp, st))
            time.sleep(0.002)
        at = [sv.submit(sp, 30, adjoint=True, ckpt_every=10) for sp in adj_specs]
        got = [sv.wait(t) for t in tickets]
        agot = [sv.wait(t) for t in at]
    for sp, st, g in zip(specs, steps, got):
        ref = _alone(sph, sp, st)
        x0 = sp["x"].astype(np.float64)
        dref = ref["x"].astype(np.float64) - x0
        assert np.linalg.norm(g["x"].astype(np.float64) - x0 - dref) <= 1e-4 * np.linalg.norm(dref)
        for k in ("v", "rho"):
            a, b = g[k].astype(np.float64), ref[k].astype(np.float64)
            assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b), k
    for sp, g in zip(adj_specs, agot):
        ref = _alone(sph, sp, 30, adjoint=True, ckpt=10)
        for k in ("x", "v", "rho", "xbar0", "vbar0", "rhobar0"):
            assert np.array_equal(g[k], ref[k]), k
        assert g["nubar"] == ref["nubar"]


def test_mixed_kinds_are_served_in_separate_batches(sph):
    """Requests of another dimension or diffusion form wait for the running batch to drain and
    then run in their own; every result is still the scene's result alone."""
    specs = [si.taylor_green_2d(24, seed=1), si.taylor_green_2d(20, seed=2, diffusion=1),
             si.taylor_green_3d(8, seed=3), si.taylor_green_2d(16, seed=4),
             si.dam_break(res=16, diffusion=1), si.dam_break(res=16, boundary=1), si.dam_break(res=20, boundary=1)]
    steps = [9, 12, 5, 7, 6, 8, 4]
    with sph.Server(8 << 30, 64) as sv:
        tickets = [sv.submit(sp, st) for sp, st in zip(specs, steps)]
        got = [sv.wait(t) for t in tickets]
    for sp, st, g in zip(specs, steps, got):
        ref = _alone(sph, sp, st)
        for k in ("x", "v", "rho"):
            assert np.array_equal(g[k], ref[k]), k


def test_an_unstable_request_fails_alone(sph):
    """A scene that goes unstable in the shared batch fails with SPH_EUNSTABLE; the scenes
    batched with it finish with their results alone."""
    good = [si.taylor_green_2d(24, seed=1), si.taylor_green_2d(20, seed=2)]
    bad = si.taylor_green_2d(16, seed=0)
    bad = dict(bad, v=(bad["v"] * 200.0).astype(np.float32))
    with sph.Server(8 << 30, 64) as sv:
        tg = [sv.submit(good[0], 30), sv.submit(bad, 40), sv.submit(good[1], 35)]
        r0 = sv.wait(tg[0])
        with pytest.raises(sph.SphError) as e:
            sv.wait(tg[1])
        assert e.value.code == sph.SPH_EUNSTABLE
        r2 = sv.wait(tg[2])
    for spec, st, g in ((good[0], 30, r0), (good[1], 35, r2)):
        ref = _alone(sph, spec, st)
        for k in ("x", "v", "rho"):
            assert np.array_equal(g[k], ref[k]), k


def test_admission_respects_budget_and_wait_is_bounded(sph):
    specs = [si.taylor_green_2d(48, seed=k) for k in range(4)]
    # budget for about one scene at a time: requests queue and run one after another
    with sph.Server(2 << 20, 16) as sv:
        tickets = [sv.submit(sp, 60) for sp in specs]
        with pytest.raises(sph.SphError) as e:
            sv.wait(tickets[-1], timeout_ms=0)
        assert e.value.code == sph.SPH_ETIMEOUT
        res = [sv.wait(t) for t in tickets]
        info = sv.stats()
    assert info["max_batch"] == 1
    t_admit = [r["t_admit"] for r in res]
    t_done = [r["t_done"] for r in res]
    assert all(t_admit[k + 1] >= t_done[k] - 1e-3 for k in range(3))
    ref = _alone(sph, specs[2], 60)
    assert np.array_equal(res[2]["x"], ref["x"])


def test_request_over_budget_is_rejected(sph):
    sp = si.taylor_green_2d(64)
    with sph.Server(1 << 20, 4) as sv:
        with pytest.raises(sph.SphError) as e:
            sv.submit(sp, 10)
        assert e.value.code == sph.SPH_EINVAL


def test_server_scenes_bypass_the_allocator_hook(sph):
    """The serving loop's scenes allocate from the CUDA stream-ordered pool, never through the
    sph_set_allocator hook (a hook may call back into an interpreter whose lock the server's
    threads would contend for): with a counting hook installed, a scene of the scene API
    allocates through it, forward and adjoint requests of the server do not."""
    import torch
    calls = [0]

    def alloc(nbytes, stream, ctx):
        calls[0] += 1
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    hooks = (sph._ALLOC_FN(alloc), sph._FREE_FN(free))
    lib = sph.lib()
    prev = sph._hooks
    assert lib.sph_set_allocator(hooks[0], hooks[1], None) == 0
    try:
        spec = si.taylor_green_2d(16, seed=0)
        with sph.scene_from(spec) as sc:  # control: the scene API allocates through the hook
            sc.step(2)
        n_scene = calls[0]
        assert n_scene > 0
        with sph.Server(1 << 30, 8) as sv:
            tf = sv.submit(spec, 6)
            ta = sv.submit(spec, 6, adjoint=True, ckpt_every=3)
            rf, ra = sv.wait(tf), sv.wait(ta)
        assert np.isfinite(rf["x"]).all() and np.isfinite(ra["vbar0"]).all()
        assert calls[0] == n_scene, f"served requests made {calls[0] - n_scene} allocations through the hook"
    finally:
        if prev is not None:
            lib.sph_set_allocator(prev[0], prev[1], None)
        else:
            lib.sph_set_allocator(sph._ALLOC_FN(), sph._FREE_FN(), None)
