"""sph_cells_noalloc: the allocation-free cell binning equals the cell structure a freshly
initialised scene builds (sph_debug_cells), call after call, whatever ran before it.

Index work, so the comparison is exact.  The file sorts last so that the GPU cases also run
after every other GPU test in one session (the static scratch then holds their leftovers)."""
import ctypes as C

import numpy as np
import pytest

import sph_inputs as si


@pytest.fixture(scope="module")
def sph():
    from paper_2507_21684_b300 import build
    build.build()
    import paper_2507_21684_b300 as m
    return m


def _shifted_tg2d():
    """Taylor-Green lattice, shuffled, with whole periods added on both axes (wrap path)."""
    s = si.taylor_green_2d(48, seed=3)
    rng = np.random.default_rng(11)
    perm = rng.permutation(s["n_fluid"])
    x = s["x"].reshape(-1, 2)[perm].copy()
    L = np.array(s["params"]["box_hi"][:2]) - np.array(s["params"]["box_lo"][:2])
    x += (rng.integers(-2, 3, size=x.shape) * L).astype(np.float32)
    s = dict(s)
    s["x"] = np.ascontiguousarray(x.astype(np.float32).reshape(s["x"].shape))
    s["v"] = np.ascontiguousarray(s["v"].reshape(-1, 2)[perm].reshape(s["v"].shape))
    s["rho"] = np.ascontiguousarray(s["rho"][perm])
    s["mass"] = np.ascontiguousarray(s["mass"][perm])
    return s


CASES = {
    "dambreak_128": lambda: si.dam_break(res=128),           # walls, closed box, two sort passes
    "tg2d_64": lambda: si.taylor_green_2d(64, seed=1),        # periodic, one sort pass
    "tg2d_48_shifted": _shifted_tg2d,                          # periodic images outside the box
    "tg3d_32": lambda: si.taylor_green_3d(32, seed=2),        # 3D, two sort passes
}


def _expected(sph, spec):
    with sph.scene_from(spec) as sc:
        start, ids = sc.debug_cells()
    return start, ids


@pytest.mark.gpu
@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_matches_scene_cells_twice(sph, case):
    import torch
    spec = CASES[case]()
    start_ref, ids_ref = _expected(sph, spec)
    d = spec["params"]["dim"]
    x = torch.from_numpy(np.ascontiguousarray(spec["x"]).reshape(-1, d)).cuda()
    n = x.shape[0]
    nc = sph.cells_noalloc(spec["params"], x, None, None)
    assert nc + 1 == start_ref.size
    stream = torch.cuda.Stream()
    for call in range(2):  # two calls in a row reuse the scratch
        start = torch.full((nc + 1,), -7, dtype=torch.int32, device="cuda")
        ids = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        assert sph.cells_noalloc(spec["params"], x, start, ids, stream=stream) == nc
        stream.synchronize()
        np.testing.assert_array_equal(start.cpu().numpy().astype(np.int64), start_ref, err_msg=f"call {call}")
        np.testing.assert_array_equal(ids.cpu().numpy(), ids_ref, err_msg=f"call {call}")


@pytest.mark.gpu
def test_noalloc_empty_and_default_stream(sph):
    import torch
    spec = si.taylor_green_2d(16, seed=0)
    x = torch.zeros((0, 2), dtype=torch.float32, device="cuda")
    nc = sph.cells_noalloc(spec["params"], x, None, None)
    start = torch.full((nc + 1,), -7, dtype=torch.int32, device="cuda")
    ids = torch.zeros((1,), dtype=torch.int32, device="cuda")
    sph.cells_noalloc(spec["params"], x, start, ids)  # legacy default stream
    torch.cuda.synchronize()
    assert int(start.abs().sum()) == 0


def test_noalloc_rejects_sizes_beyond_scratch_without_device(sph):
    spec = si.taylor_green_2d(16, seed=0)
    L = sph.lib()
    pp = sph.Params.from_dict(spec["params"])
    nc = C.c_int32(0)
    rc = L.sph_cells_noalloc(C.byref(pp), None, sph.NOALLOC_MAX_PARTICLES + 1, None, 0, None, C.byref(nc), None)
    assert rc == sph.SPH_EINVAL
    assert b"static scratch" in L.sph_last_error()
    # a short cell_start is rejected before anything is enqueued, and n_cells is reported
    rc = L.sph_cells_noalloc(C.byref(pp), None, 0, None, 0, None, C.byref(nc), None)
    assert rc == sph.SPH_EINVAL and nc.value > 0
    assert b"n_cells + 1" in L.sph_last_error()
