"""Pins of the oracle's smoothing kernels (the paper names none; Sec. 2.1),
in three dimensions and in one (the 1D Sod problem of Sec. 3).

Each pin is independent of the oracle's own formulas: quadrature of the
normalisation integral, finite differences of W, the published central
values sigma / h^D, compact support and smoothness at the joins.
"""
import math

import numpy as np
import pytest

KERNELS = [0, 1, 2]
DIMS = [3, 1]
# published central values: sigma for D = 3 (M4, Wendland C2, C4) and the 1D
# ones, 2/3 for M4 and (5/4, 3/2) / 2 for the Wendland functions of support 2h
SIGMA = {(0, 3): 1.0 / math.pi, (1, 3): 21.0 / (16.0 * math.pi), (2, 3): 495.0 / (256.0 * math.pi),
         (0, 1): 2.0 / 3.0, (1, 1): 5.0 / 8.0, (2, 1): 3.0 / 4.0}


@pytest.mark.parametrize("dim", DIMS)
@pytest.mark.parametrize("k", KERNELS)
@pytest.mark.parametrize("h", [0.3, 1.0, 2.5])
def test_normalisation(orc, k, h, dim):
    """Integral of W over space is 1 (radial quadrature on [0, 2h]: weight
    4 pi r^2 in 3D, 2 in 1D).  Every kernel is a polynomial in r on [0, h]
    and on [h, 2h], so 20-point Gauss-Legendre on each piece (exact to degree
    39) gives the integral to rounding."""
    W = orc.lib().orc_W
    wt = (lambda r: 4.0 * math.pi * r * r) if dim == 3 else (lambda r: 2.0)
    x, wq = np.polynomial.legendre.leggauss(20)
    val = 0.0
    for a, b in ((0.0, h), (h, 2.0 * h)):
        r = 0.5 * (b - a) * x + 0.5 * (a + b)
        val += 0.5 * (b - a) * sum(wi * wt(ri) * W(k, dim, ri, h) for ri, wi in zip(r, wq))
    assert abs(val - 1.0) < 1e-12


@pytest.mark.parametrize("dim", DIMS)
@pytest.mark.parametrize("k", KERNELS)
def test_central_value(orc, k, dim):
    """W(0, h) = sigma / h^D with the published normalisation constants."""
    for h in (0.5, 1.0, 2.0):
        assert orc.lib().orc_W(k, dim, 0.0, h) == pytest.approx(SIGMA[(k, dim)] / h ** dim, rel=1e-15)


@pytest.mark.parametrize("dim", DIMS)
@pytest.mark.parametrize("k", KERNELS)
def test_dWdr_matches_finite_difference(orc, k, dim):
    h = 0.7
    r = np.linspace(0.01, 1.99, 397) * h
    eps = 1e-6 * h
    Wp, _, _ = orc.kernel(k, r + eps, h, dim)
    Wm, _, _ = orc.kernel(k, r - eps, h, dim)
    _, dr, _ = orc.kernel(k, r, h, dim)
    fd = (Wp - Wm) / (2 * eps)
    scale = np.abs(dr).max()
    assert np.max(np.abs(fd - dr)) < 1e-7 * scale


@pytest.mark.parametrize("dim", DIMS)
@pytest.mark.parametrize("k", KERNELS)
def test_dWdh_matches_finite_difference(orc, k, dim):
    h = 0.7
    r = np.linspace(0.0, 1.99, 400) * h
    eps = 1e-6 * h
    Wp, _, _ = orc.kernel(k, r, h + eps, dim)
    Wm, _, _ = orc.kernel(k, r, h - eps, dim)
    _, _, dh = orc.kernel(k, r, h, dim)
    fd = (Wp - Wm) / (2 * eps)
    scale = np.abs(dh).max()
    assert np.max(np.abs(fd - dh)) < 1e-7 * scale


@pytest.mark.parametrize("dim", DIMS)
@pytest.mark.parametrize("k", KERNELS)
def test_compact_support_and_smooth_edge(orc, k, dim):
    h = 1.3
    W, dr, dh = orc.kernel(k, np.array([2 * h, 2.5 * h, 10 * h]), h, dim)
    assert np.all(W == 0) and np.all(dr == 0) and np.all(dh == 0)
    # W and dW/dr vanish continuously at r -> 2h
    W, dr, _ = orc.kernel(k, np.array([2 * h * (1 - 1e-5)]), h, dim)
    assert abs(W[0]) < 1e-13 and abs(dr[0]) < 1e-8


def test_m4_join_is_smooth(orc):
    """M4 cubic spline: value, first and second derivative continuous at q = 1."""
    h = 1.0
    e = 1e-7
    W, dr, _ = orc.kernel(0, np.array([1 - e, 1 + e]), h)
    # the jump left after removing the linear change across the join
    assert abs((W[1] - W[0]) - e * (dr[0] + dr[1])) < 1e-12
    assert abs(dr[0] - dr[1]) < 1e-6
    _, d1, _ = orc.kernel(0, np.array([1 - 2e-4, 1 - 1e-4, 1 + 1e-4, 1 + 2e-4]), h)
    # a jump in the second derivative would leave O(1e-4) here, smooth leaves O(1e-8)
    assert abs((d1[1] - d1[0]) - (d1[3] - d1[2])) < 1e-7


@pytest.mark.parametrize("k", KERNELS)
def test_kernel_is_decreasing(orc, k):
    r = np.linspace(0, 2, 2001)
    W, dr, _ = orc.kernel(k, r, 1.0)
    assert np.all(np.diff(W) <= 1e-15)
    assert np.all(dr <= 0)
