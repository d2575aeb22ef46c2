"""Oracle kernel functions pinned to the paper's printed constants and to calculus (App. A.1)."""
import math
from pathlib import Path

import numpy as np
import pytest
from scipy import integrate

from tests.scenes import params

GOLDEN = Path(__file__).parent / "golden" / "kernel_scales.txt"


def _rows():
    for line in GOLDEN.read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            d, cd, expr, scale = line.split()
            cd_expr = eval(expr, {"__builtins__": {}}, {"pi": math.pi})
            assert abs(float(cd) - cd_expr) < 1e-12
            yield int(d), cd_expr, float(scale)


@pytest.mark.parametrize("dim,kern", [(2, 0), (3, 0), (2, 1), (3, 1)])
def test_kernel_integrates_to_one(orc, dim, kern):
    area = 2 * math.pi if dim == 2 else 4 * math.pi
    f = lambda q: orc.kernel(dim, kern, q)[0] * orc.kernel(dim, kern, q)[3] * area * q ** (dim - 1)
    val, _ = integrate.quad(f, 0.0, 1.0, epsabs=1e-14, epsrel=1e-13)
    assert abs(val - 1.0) < 1e-12


def test_wendland4_printed_constants_and_scales(orc):
    """C_d and H/h of the Wendland-4 kernel as printed in App. A.1 (tests/golden)."""
    for dim, cd_printed, scale_printed in _rows():
        cd = orc.kernel(dim, 0, 0.0)[3]
        assert abs(cd - cd_printed) < 1e-12
        area = 2 * math.pi if dim == 2 else 4 * math.pi
        m2, _ = integrate.quad(lambda q: cd * orc.kernel(dim, 0, q)[0] * area * q ** (dim + 1), 0, 1,
                               epsabs=1e-15, epsrel=1e-13)
        sigma = math.sqrt(m2 / dim)
        assert abs(1.0 / (2.0 * sigma) - scale_printed) < 2e-6


@pytest.mark.parametrize("dim,kern", [(2, 0), (3, 0), (3, 1)])
def test_kernel_derivatives_match_finite_differences(orc, dim, kern):
    for q in np.linspace(0.05, 0.95, 19):
        w, w1, w2, _ = orc.kernel(dim, kern, q)
        h = 1e-6
        wp, wm = orc.kernel(dim, kern, q + h)[0], orc.kernel(dim, kern, q - h)[0]
        w1p, w1m = orc.kernel(dim, kern, q + h)[1], orc.kernel(dim, kern, q - h)[1]
        assert abs((wp - wm) / (2 * h) - w1) < 1e-7
        assert abs((w1p - w1m) / (2 * h) - w2) < 1e-6
    # compact support, smooth zero at q = 1
    assert orc.kernel(dim, kern, 1.0)[:3] == (0.0, 0.0, 0.0)


@pytest.mark.parametrize("dim,kern", [(2, 0), (3, 0), (3, 1)])
def test_gradient_is_fd_of_W(orc, dim, kern):
    H = 0.1
    p = params(dim=dim, kernel=kern, H=H)
    rng = np.random.default_rng(1)
    for _ in range(20):
        r = rng.uniform(-H, H, dim)
        if np.linalg.norm(r) > 0.98 * H or np.linalg.norm(r) < 0.05 * H:
            continue
        _, G = orc.kernel_eval(p, r)
        fd = np.zeros(dim)
        for k in range(dim):
            e = np.zeros(dim)
            e[k] = 1e-7
            fd[k] = (orc.kernel_eval(p, r + e)[0] - orc.kernel_eval(p, r - e)[0]) / 2e-7
        assert np.allclose(G, fd, rtol=1e-6, atol=1e-6 * np.abs(G).max())
    W0, G0 = orc.kernel_eval(p, np.zeros(dim))
    assert np.all(G0 == 0.0) and W0 > 0
