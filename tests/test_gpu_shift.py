"""CUDA path of the explicit particle shifting (end of each step) vs the FP64 oracle.

The shift of one step is compared as the difference between a shifted and an unshifted GPU
step against the oracle's displacement at the unshifted GPU result; rollouts with shifting
(eager, graph-captured with a Verlet skin, free surface and walls, 3D) are compared with the
oracle's rollouts at the 10-step bar of 1e-3."""
import numpy as np
import pytest

import sph_inputs as si
from tests.test_gpu_parity import check_rollout, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    from paper_2507_21684_b300 import build
    build.build()
    import paper_2507_21684_b300 as m
    return m


def _with(s, **kw):
    return dict(s, params=dict(s["params"], **kw))


ONE_STEP = {
    "tgv2d_64": lambda: si.taylor_green_2d(64, seed=3, jitter=0.2, shift=0.1),
    "dambreak_64": lambda: si.dam_break(res=64, shift=0.05),
    "tgv3d_24": lambda: si.taylor_green_3d(24, seed=1, jitter=0.2, shift=0.1),
}


@pytest.mark.parametrize("case", list(ONE_STEP))
def test_one_step_shift_matches_oracle(sph, orc, case):
    s = ONE_STEP[case]()
    s0 = _with(s, shift=0.0)
    with sph.scene_from(s0) as sc:
        sc.set_execution(False)
        sc.step(1)
        x0, v0, r0 = sc.get_state()
    with sph.scene_from(s) as sc:
        sc.set_execution(False)
        sc.step(1)
        x1, v1, r1 = sc.get_state()
    # the shift moves positions only
    assert np.array_equal(v1, v0) and np.array_equal(r1, r0)
    nf = s["n_fluid"]
    d_gpu = x1[:nf].astype(np.float64) - x0[:nf]
    d_orc, lam = orc.shift(dict(s, x=x0, v=v0, rho=r0))
    assert np.abs(d_orc).max() > 0
    # float32 positions: each difference carries up to one ulp of x
    ulp = np.spacing(np.abs(x0[:nf]).astype(np.float32)).astype(np.float64)
    band = (lam > 0.4 - 1e-4) & (lam < 0.4 + 1e-4) | (lam > 0.75 - 1e-4) & (lam < 0.75 + 1e-4)
    err = np.abs(d_gpu - d_orc)[~band]
    assert np.all(err <= 2e-3 * np.abs(d_orc).max() + 1.5 * ulp[~band]), (err.max(), np.abs(d_orc).max())
    assert rel(d_gpu, d_orc) < 1e-3
    assert np.array_equal(x1[nf:], x0[nf:])  # walls stay


ROLL = {
    "tgv2d_64_eager": (lambda: si.taylor_green_2d(64, seed=0, jitter=0.2, shift=0.1), False),
    "tgv2d_64_graph_skin": (lambda: si.taylor_green_2d(64, seed=0, jitter=0.2, shift=0.1, skin=0.1 / 64 * 4,
                                                       rebuild_interval=1 << 20), True),
    "dambreak_128": (lambda: si.dam_break(res=128, shift=0.05), True),
    "dambreak_64_skin": (lambda: si.dam_break(res=64, shift=0.05, skin=float(np.float32(0.02 * 4 / 64)),
                                              rebuild_interval=1 << 20), True),
    "tgv3d_24": (lambda: si.taylor_green_3d(24, seed=1, jitter=0.2, shift=0.1), True),
    # 3D with a Verlet skin: the sweep's and the shift's rebuilds in conditional graph nodes, with
    # x sub-bins, and the renormalised diffusion's gradient pass
    "tgv3d_24_renorm_skin": (lambda: si.taylor_green_3d(24, seed=1, jitter=0.2, shift=0.1, diffusion=1,
                                                        skin=float(np.float32(0.1 * 2.43 / 24)),
                                                        rebuild_interval=1 << 20), True),
}


@pytest.mark.parametrize("case", list(ROLL))
def test_ten_step_rollout_with_shifting(sph, orc, case):
    make, graphs = ROLL[case]
    s = make()
    with sph.scene_from(s) as sc:
        sc.set_execution(graphs)
        sc.step(10)
        x, v, rho = sc.get_state()
    xo, vo, ro = orc.rollout(s, 10)
    check_rollout(s, 10, x, v, rho, xo, vo, ro)


def test_shifting_with_skin_rebuilds_and_matches_eager(sph, orc):
    """200 graph-captured steps with a Verlet skin (rebuilds decided on the device, before the
    sweep and again before the shift) against eager steps that rebuild twice per step."""
    s = si.taylor_green_2d(48, seed=2, jitter=0.2, shift=0.1, skin=float(np.float32(0.1 * 4 / 48)),
                           rebuild_interval=1 << 20)
    with sph.scene_from(s) as sc:
        sc.step(200)
        st = sc.stats()
        xg, vg, rg = sc.get_state()
    with sph.scene_from(s) as sc:
        sc.set_execution(False)
        sc.step(200)
        xe, ve, re_ = sc.get_state()
    assert 0 < st["rebuilds"] < 200
    x0 = s["x"].astype(np.float64)
    assert rel(xg - x0, xe - x0) < 1e-3
    assert rel(vg, ve) < 1e-3


def test_shifting_rejects_rollout_and_mixed_batches(sph):
    s = si.taylor_green_2d(16, seed=0, shift=0.1)
    with sph.scene_from(s) as sc:
        with pytest.raises(Exception, match="shifting"):
            sc.rollout(4, 2)
    with pytest.raises(Exception, match="shifting"):
        sph.Scene.batch([s, si.taylor_green_2d(16, seed=1)])


def test_shifting_batch_bitwise_equal_alone(sph):
    specs = [si.dam_break(res=32, shift=0.05), si.taylor_green_2d(24, seed=3, jitter=0.2, shift=0.1),
             si.dam_break(res=40, shift=0.02)]
    with sph.Scene.batch(specs) as bt:
        bt.step(9)
        xb, vb, rb = bt.get_state()
        rows = list(zip(bt.first_row, bt.rows))
    for spec, (f, n) in zip(specs, rows):
        with sph.scene_from(spec) as sc:
            sc.step(9)
            x, v, r = sc.get_state()
        assert np.array_equal(x, xb[f:f + n]) and np.array_equal(v, vb[f:f + n]) and np.array_equal(r, rb[f:f + n])
