"""Tile-shape variants of the library (threads per particle, targets per tile) give the oracle's
results too, and the autotuner that picks among them runs each in its own process."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import sph_inputs as si
from tests.test_gpu_parity import check_rollout

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_2507_21684_b300.build import VARIANTS as _VARIANTS  # noqa: E402  (no compilation at import)
SCRIPT = r"""
import sys, numpy as np
import paper_2507_21684_b300 as sph
from paper_2507_21684_b300 import tune
spec = tune.load_spec(sys.argv[1])
with sph.scene_from(spec) as sc:
    sc.step(10)
    x, v, r = sc.get_state()
np.savez(sys.argv[2], x=x, v=v, rho=r)
"""


@pytest.mark.parametrize("variant", sorted(v for v in _VARIANTS if v != "default"))
@pytest.mark.parametrize("case", ["dambreak_64", "tgv3d_24"])
def test_variant_rollouts_match_oracle(orc, tmp_path, variant, case):
    from paper_2507_21684_b300 import build, tune
    if variant not in tune.shape_variants(2 if case == "dambreak_64" else 3):
        pytest.skip("the variant runs the default shape in this dimension")
    build.build(variant=variant)
    s = si.dam_break(res=64) if case == "dambreak_64" else si.taylor_green_3d(24, seed=1)
    spec, out = str(tmp_path / "s.npz"), str(tmp_path / "o.npz")
    tune.save_spec(s, spec)
    subprocess.run([sys.executable, "-c", SCRIPT, spec, out], cwd=ROOT, check=True,
                   env=dict(os.environ, SPH_B300_VARIANT=variant))
    z = np.load(out)
    xo, vo, ro = orc.rollout(s, 10)
    check_rollout(s, 10, z["x"], z["v"], z["rho"], xo, vo, ro)


def test_tile_tuner_times_every_variant():
    from paper_2507_21684_b300 import build, tune
    r = tune.tune_tiles(si.dam_break(res=32), steps=20, warmup=5)
    assert {t["variant"] for t in r["table"]} == set(tune.shape_variants(2))
    assert r["variant"] in build.VARIANTS and all(t["ms_per_step"] > 0 for t in r["table"])


def test_cooperative_3d_rebuild_with_a_skin_matches_oracle(orc, tmp_path):
    """The library variant whose captured 3D steps rebuild in one cooperative launch (keys with x
    sub-bins computed in its first sort pass, the sub-bins' offsets written by its permute) gives
    the oracle's 3D rollout under a Verlet skin, rebuilding fewer times than it steps."""
    from paper_2507_21684_b300 import build, tune
    build.build(variant="coop3")
    s = si.taylor_green_3d(24, seed=3)
    p = dict(s["params"], skin=float(np.float32(0.1 * s["params"]["H"])), rebuild_interval=1 << 20)
    s = dict(s, params=p)
    spec, out = str(tmp_path / "s.npz"), str(tmp_path / "o.npz")
    tune.save_spec(s, spec)
    script = SCRIPT.replace("sc.step(10)", "sc.step(40)\n    st = sc.stats()").replace(
        "np.savez(sys.argv[2], x=x, v=v, rho=r)", "np.savez(sys.argv[2], x=x, v=v, rho=r, rebuilds=st['rebuilds'])")
    subprocess.run([sys.executable, "-c", script, spec, out], cwd=ROOT, check=True,
                   env=dict(os.environ, SPH_B300_VARIANT="coop3"))
    z = np.load(out)
    assert 1 < int(z["rebuilds"]) < 40
    xo, vo, ro = orc.rollout(s, 40)
    check_rollout(s, 40, z["x"], z["v"], z["rho"], xo, vo, ro)
