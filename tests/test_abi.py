"""The C-ABI library loads and exports every entry point include/*.h declares (no GPU needed)."""
import ctypes as C
import re
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]


def _declared():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        for m in re.finditer(r"SPH_API\s+[\w\s\*]+?\b(sph_\w+)\s*\(", h.read_text()):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    from paper_2507_21684_b300 import build
    build.build()
    import paper_2507_21684_b300 as sph
    return sph.lib()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("sph_init", "sph_step", "sph_rollout", "sph_adjoint", "sph_get_state", "sph_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    for name in _declared():
        assert hasattr(L, name), name


def test_abi_version_and_error_string(L):
    assert L.sph_abi_version() == 2
    assert isinstance(L.sph_last_error(), bytes)


def test_invalid_parameters_rejected_without_device(L):
    import paper_2507_21684_b300 as sph
    import sph_inputs as si
    s = si.taylor_green_2d(8)
    p = dict(s["params"])
    p["H"] = 0.5  # only one cell of edge >= H per periodic axis
    with pytest.raises(sph.SphError) as e:
        sph.Scene(p, s["n_fluid"], 0, s["x"], s["v"], s["rho"], s["mass"])
    assert e.value.code == sph.SPH_EINVAL
    p = dict(s["params"])
    p["dim"] = 4
    with pytest.raises(sph.SphError) as e:
        sph.Scene(p, s["n_fluid"], 0, s["x"], s["v"], s["rho"], s["mass"])
    assert e.value.code == sph.SPH_EINVAL


def test_tile_tuner_candidates_per_dimension():
    """The tuner times, for a scene, the default library and every variant that changes the tile
    shape of the scene's dimension (a variant of the other dimension's shape would time the
    default shape again)."""
    from paper_2507_21684_b300 import build, tune
    for dim in (2, 3):
        c = tune.shape_variants(dim)
        assert c[0] == "default" and len(set(c)) == len(c)
        for v, d in build.VARIANTS.items():
            if v != "default":
                assert (v in c) == any(k.startswith(f"SPH_TILE{dim}_") or k == f"SPH_W{dim}" or
                                       (dim == 3 and k.startswith("SPH_W_")) for k in d)
    assert "small" in tune.shape_variants(2) and "small" not in tune.shape_variants(3)
    assert "small3" in tune.shape_variants(3) and "small3" not in tune.shape_variants(2)
    # the staged 3D traversal is a candidate against the warp-per-tile one in 3D only
    assert "staged3" in tune.shape_variants(3) and "staged3" not in tune.shape_variants(2)


def test_combined_variant_names():
    """A 3D and a 2D choice combine into one library; conflicting choices are refused."""
    from paper_2507_21684_b300 import build
    assert build.canonical("small+default") == "small"
    assert build.canonical("small+small3") == build.canonical("small3+small") == "small+small3"
    assert build.lib_path("small3+small").name == "libsph_b300_small_small3.so"
    m = build.variant_macros("small+staged3")
    assert m["SPH_W3"] == 0 and m["SPH_TILE2_TP"] == 32
    with pytest.raises(ValueError):
        build.variant_macros("lanes8+small")  # both set the 2D shape
    with pytest.raises(ValueError):
        build.canonical("nosuch")
