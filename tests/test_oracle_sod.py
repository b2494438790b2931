"""Pins of the oracle in one dimension (the Sod shock tube of Sec. 3).

Independent checks: the density of a uniform 1D lattice with the M4 kernel
(the cubic B-spline of knot spacing h) from Poisson summation,
rho = (m/dx) (1 + 2 sum_n sinc^4(pi n h/dx)); the 1D law h = eta m / rho at
convergence; the neighbour count 4 eta of a uniform line; and the
conservation identities (sum m a = 0, sum m (v.a + du/dt) = 0) on the Sod
initial state with random velocities.
"""
import math

import numpy as np
import pytest

from helpers import oracle_params
from paper_2007_03097_gb300 import inputs


def _line(n, L=2.0, eta=1.2, kernel=0, fixed_h=True):
    """Uniform periodic line of n particles on [0, L), total mass 1."""
    w = inputs.sod(100, kernel=kernel, eta=eta)
    dx = L / n
    x = (np.arange(n) + 0.5) * dx
    w = w.subset(np.zeros(n, dtype=np.int64))
    w.x = x
    w.m[:] = 1.0 / n
    w.h[:] = eta * dx
    w.u[:] = 1.0
    w.params.update(fixed_h=fixed_h)
    return w, dx


@pytest.mark.parametrize("eta", [1.2, 1.37, 2.05])
def test_uniform_line_density_from_poisson_sum(orc, eta):
    w, dx = _line(1000, eta=eta)
    d = orc.density(oracle_params(orc, w), w.x, w.y, w.z, w.m, w.h)
    n = np.arange(1, 200001, dtype=np.float64)
    s = np.sin(math.pi * n * eta) / (math.pi * n * eta)
    ref = (w.m[0] / dx) * (1.0 + 2.0 * np.sum(s ** 4))
    assert np.max(np.abs(d.rho / ref - 1)) < 1e-12
    # neighbours within 2h on a uniform line: 2 floor(2 eta) (strictly inside)
    assert np.all(d.nnb == 2 * int(math.floor(2 * eta - 1e-12)))


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_h_law_at_convergence_in_1d(orc, kernel):
    w = inputs.sod(400, kernel=kernel)
    p = oracle_params(orc, w)
    d = orc.density(p, w.x, w.y, w.z, w.m, w.h)
    assert d.status == 0
    # Eq. 9 with D = 1: h = eta m / rho
    assert np.max(np.abs(d.h - p.eta * w.m / d.rho) / d.h) < 1e-10
    # far from the interfaces the density is the state's own, up to the
    # lattice (aliasing) error of each kernel at eta = 1.2 (0.3 % for the
    # 1D Wendland C2)
    left = (w.x > 0.1) & (w.x < 0.4)
    right = (w.x > 0.7) & (w.x < 1.3)
    assert np.max(np.abs(d.rho[left] / 1.0 - 1)) < 5e-3
    assert np.max(np.abs(d.rho[right] / 0.125 - 1)) < 5e-3


def test_conservation_in_1d(orc):
    w = inputs.sod(600, kernel=1)
    rng = np.random.default_rng(4)
    w.vx = 0.3 * rng.standard_normal(w.n)
    p = oracle_params(orc, w)
    d = orc.density(p, w.x, w.y, w.z, w.m, w.h)
    P, c = orc.eos(p.gamma, d.rho, w.u)
    f = orc.forces(p, w.x, w.y, w.z, w.vx, w.vy, w.vz, w.m, d.h, d.rho, P, c)
    eps = np.finfo(np.float64).eps
    assert abs(np.sum(w.m * f.ax)) < 10 * eps * np.sum(w.m * f.S_a)
    assert np.all(f.ay == 0) and np.all(f.az == 0)
    power = np.sum(w.m * (w.vx * f.ax + f.dudt))
    assert abs(power) < 10 * eps * np.sum(w.m * (np.abs(w.vx) * f.S_a + f.S_u))
    assert np.max(np.abs(f.ax)) > 0


def _golden_sod():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sod_initial_state.txt")
    rows = {}
    with open(path) as f:
        for line in f:
            t = line.split()
            if t and not t[0].startswith("#"):
                rows[t[0]] = [float(v) for v in t[1:]]
    return rows


def test_sod_state_is_the_papers(orc):
    """The workload's two states are those printed in Sec. 3
    (tests/golden/sod_initial_state.txt), and the oracle reads them back from
    the particles: density from the summation (up to the lattice error of M4
    at eta = 1.2), velocity zero, and pressure from the EOS P = (gamma-1) rho u."""
    g = _golden_sod()
    assert tuple(g["left"][2:]) == inputs.SOD_LEFT and tuple(g["right"][2:]) == inputs.SOD_RIGHT
    w = inputs.sod(int(g["particles"][0]) // 10)
    p = oracle_params(orc, w)
    d = orc.density(p, w.x, w.y, w.z, w.m, w.h)
    P, _ = orc.eos(p.gamma, d.rho, w.u)
    for side in ("left", "right"):
        x0, x1, rho, v, pr = g[side]
        inner = (w.x > x0 + 0.1) & (w.x < x1 - 0.1)
        assert inner.sum() > 50
        assert np.max(np.abs(d.rho[inner] / rho - 1)) < 5e-3
        assert np.max(np.abs(P[inner] / pr - 1)) < 5e-3
        assert np.all(w.vx[inner] == v)
    # at full size the tube holds the paper's particle count, up to rounding
    # the two states' counts to a spacing ratio of 8 (8,888 + 1,111)
    w = inputs.sod(int(g["particles"][0]))
    assert abs(np.count_nonzero(w.x < 1.0) - int(g["particles"][0])) <= 1
