"""sph_cells_noalloc: the allocation-free cell binning equals the cell structure a freshly
initialised scene builds (sph_debug_cells) and the FP64 oracle's cells, call after call, whatever
ran before it, up to the size of its static scratch, and without taking device memory.

Index work, so the comparison is exact.  The file sorts last so that the GPU cases also run
after every other GPU test in one session (the static scratch then holds their leftovers)."""
import ctypes as C

import numpy as np
import pytest

import oracle as orc
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


def _random_2d(n: int, cells_per_axis: int = 512, seed: int = 5):
    """n uniform random particles in the unit square binned on a cells_per_axis^2 grid (18 key
    bits, three sort passes), x periodic and y closed, some particles placed outside the box on
    both axes (wrapped in x, clamped to the edge cells in y)."""
    s = si.taylor_green_2d(16, seed=0)
    p = dict(s["params"], H=float(np.float32(1.0 / cells_per_axis)), skin=0.0, periodic_mask=1)
    ids = np.arange(n)
    x = np.stack([si.uniform24(seed, 7, ids, 0), si.uniform24(seed, 7, ids, 1)], 1).astype(np.float64)
    out = si.uniform24(seed, 8, ids, 0) < 0.02
    x[out] += (si.uniform24(seed, 8, ids[out], 1)[:, None] * 2.0 - 1.0) * 1.5
    x = np.ascontiguousarray(x.astype(np.float32))
    z = np.zeros_like(x)
    return dict(params=p, n_fluid=n, n_wall=0, x=x, v=z, rho=np.ones(n, np.float32),
                mass=np.ones(n, np.float32))


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


def _oracle_cells(spec):
    d = spec["params"]["dim"]
    _, _, ids, start = orc.cells(spec["params"], np.ascontiguousarray(spec["x"]).reshape(-1, d))
    return start, ids


def _no_device_allocation(torch, fn):
    """Run fn (which enqueues one call and synchronises) and check that neither the device's free
    memory nor the caching allocator's allocation count moved."""
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    n0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    fn()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    n1 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    assert free1 == free0, f"device free memory moved by {free0 - free1} bytes"
    assert n1 == n0, "the caching allocator served an allocation during the call"


@pytest.mark.gpu
@pytest.mark.parametrize("case", list(CASES))
def test_noalloc_matches_scene_cells_twice(sph, case):
    import torch
    spec = CASES[case]()
    start_ref, ids_ref = _expected(sph, spec)
    o_start, o_ids = _oracle_cells(spec)
    np.testing.assert_array_equal(start_ref, o_start)
    np.testing.assert_array_equal(ids_ref, o_ids)
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
@pytest.mark.parametrize("n", [200_000, 524_288])
def test_noalloc_large_three_passes_no_allocation(sph, n):
    """Three sort passes over a 512 x 512 grid (the multi-block histogram scan), up to exactly
    SPH_NOALLOC_MAX_PARTICLES (the histogram fills the static scratch); outputs equal the oracle's
    cells on both calls, and the second call takes no device memory."""
    import torch
    assert n <= sph.NOALLOC_MAX_PARTICLES
    spec = _random_2d(n)
    o_start, o_ids = _oracle_cells(spec)
    x = torch.from_numpy(spec["x"]).cuda()
    nc = sph.cells_noalloc(spec["params"], x, None, None)
    assert nc == 512 * 512 and nc + 1 == o_start.size
    start = torch.empty((nc + 1,), dtype=torch.int32, device="cuda")
    ids = torch.empty((n,), dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    for call in range(2):
        start.fill_(-7)
        ids.fill_(-7)

        def one():
            assert sph.cells_noalloc(spec["params"], x, start, ids, stream=stream) == nc
            stream.synchronize()
        if call == 0:
            one()  # the first call may load kernels lazily
        else:
            _no_device_allocation(torch, one)
        np.testing.assert_array_equal(start.cpu().numpy().astype(np.int64), o_start, err_msg=f"call {call}")
        np.testing.assert_array_equal(ids.cpu().numpy(), o_ids, err_msg=f"call {call}")


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


def test_noalloc_wrapper_rejects_bad_buffers(sph):
    """The binding refuses host, mistyped, strided or short buffers before calling the library."""
    torch = pytest.importorskip("torch")
    spec = si.taylor_green_2d(16, seed=0)
    with pytest.raises(ValueError):
        sph.cells_noalloc(spec["params"], torch.zeros((4, 2), dtype=torch.float32), None, None)
    with pytest.raises(ValueError):
        sph.cells_noalloc(spec["params"], np.zeros((4, 2), np.float32), None, None)
    if not torch.cuda.is_available():
        return
    x = torch.zeros((8, 2), dtype=torch.float32, device="cuda")
    nc = sph.cells_noalloc(spec["params"], x, None, None)
    good_s = torch.zeros((nc + 1,), dtype=torch.int32, device="cuda")
    good_i = torch.zeros((8,), dtype=torch.int32, device="cuda")
    bad = [
        (x.double(), good_s, good_i),
        (torch.zeros((8, 3), dtype=torch.float32, device="cuda"), good_s, good_i),
        (torch.zeros((2, 8), dtype=torch.float32, device="cuda").t(), good_s, good_i),
        (x, good_s[:-1], good_i),
        (x, good_s.long(), good_i),
        (x, good_s, good_i[:-1]),
        (x, good_s, good_i.long()),
        (x, good_s, torch.zeros((16,), dtype=torch.int32, device="cuda")[::2]),
    ]
    for xx, ss, ii in bad:
        with pytest.raises(ValueError):
            sph.cells_noalloc(spec["params"], xx, ss, ii)
