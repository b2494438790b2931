"""Pins of the oracle's density sum (Eq. 7) and h-rho fixed point (Eq. 9).

Independent checks: a perfect periodic lattice summed over integer lattice
offsets (no particles, no minimum image), the fixed-point identity
h = eta (m/rho)^(1/3), an independent bracketing root finder (Brent) on the
same equation, the expected neighbour count (32 pi / 3) eta^3 of a uniform
medium, and the failure flags.
"""
import itertools
import math

import numpy as np
import pytest
from scipy.optimize import brentq

from paper_2007_03097_gb300 import inputs


from helpers import oracle_params as _params  # noqa: E402


def _unused_params(orc, w, **kw):
    p = dict(w.params)
    p.update(kw)
    keys = {f for f in orc.Params.__dataclass_fields__}
    return orc.Params(**{k: v for k, v in p.items() if k in keys})


@pytest.mark.parametrize("k", [0, 1, 2])
def test_perfect_lattice_equals_offset_sum(orc, k):
    n_side, hf = 12, 1.3
    w = inputs.lattice(n_side, jitter=0.0, kernel=k, h_factor=hf)
    p = _params(orc, w, fixed_h=True)
    d = orc.density(p, w.x, w.y, w.z, w.m, w.h)
    dx = 1.0 / n_side
    h = hf * dx
    rng = range(-3, 4)
    offs = np.array([math.sqrt(a * a + b * b + c * c) * dx for a, b, c in itertools.product(rng, rng, rng)])
    W, _, _ = orc.kernel(k, offs, h)
    ref = (1.0 / w.n) * np.sum(W[offs < 2 * h])
    assert np.max(np.abs(d.rho / ref - 1)) < 1e-13
    cnt = int(np.sum((offs < 2 * h) & (offs > 0)))
    assert np.all(d.nnb == cnt)


def test_large_h_recovers_mean_density(orc):
    w = inputs.lattice(10, jitter=0.1, kernel=2, h_factor=2.2)
    d = orc.density(_params(orc, w, fixed_h=True), w.x, w.y, w.z, w.m, w.h)
    assert abs(d.rho.mean() - 1.0) < 5e-3


def _sedov_small(n_side=10):
    return inputs.sedov(n_side)


def test_fixed_point_identity_and_neighbour_count(orc):
    w = _sedov_small(10)
    p = _params(orc, w)
    d = orc.density(p, w.x, w.y, w.z, w.m, w.h * 1.07)
    assert d.status == 0
    assert np.all(d.flags == orc.DONE)
    resid = np.abs(d.h - p.eta * (w.m / d.rho) ** (1 / 3)) / d.h
    assert resid.max() < 1e-10
    nbar = 32 * math.pi / 3 * p.eta ** 3
    assert abs(d.nnb.mean() / nbar - 1) < 0.05
    assert d.sweeps.min() >= 2


def test_newton_root_matches_brent(orc):
    w = _sedov_small(8)
    p = _params(orc, w)
    d = orc.density(p, w.x, w.y, w.z, w.m, w.h)
    pf = _params(orc, w, fixed_h=True)
    eta3 = p.eta ** 3
    for a in (0, 17, 200, 511):
        def g(h):
            hh = w.h.copy()
            hh[a] = h
            r = orc.density(pf, w.x, w.y, w.z, w.m, hh, targets=[a]).rho[a]
            return w.m[a] * eta3 / h ** 3 - r
        root = brentq(g, 0.5 * d.h[a], 2.0 * d.h[a], xtol=1e-15, rtol=1e-14)
        assert abs(root / d.h[a] - 1) < 1e-10


def test_targets_subset_matches_full(orc):
    w = _sedov_small(8)
    p = _params(orc, w)
    full = orc.density(p, w.x, w.y, w.z, w.m, w.h)
    t = np.array([3, 99, 400])
    sub = orc.density(p, w.x, w.y, w.z, w.m, w.h, targets=t)
    assert np.array_equal(sub.h[t], full.h[t]) and np.array_equal(sub.rho[t], full.rho[t])


def test_failure_flags(orc):
    w = _sedov_small(6)
    p = _params(orc, w, max_sweeps=2)
    d = orc.density(p, w.x, w.y, w.z, w.m, w.h * 3.0)
    assert d.status & orc.NOT_CONVERGED
    assert np.all(d.flags & orc.NOT_CONVERGED)
    p = _params(orc, w, h_max=0.5 * w.h[0])
    d = orc.density(p, w.x, w.y, w.z, w.m, w.h * 0.4)
    assert d.status & orc.H_BOUNDS
    assert np.all(d.h <= 0.5 * w.h[0])
