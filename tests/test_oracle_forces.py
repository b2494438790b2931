"""Pins of the oracle's force pass (Eqs. 5-6, Monaghan viscosity).

Independent checks: exact semi-discrete momentum and energy conservation
(pair antisymmetry; the energy identity holds for any rho, with or without
viscosity), zero force on a perfect lattice at rest, the continuum limits
a = -grad P / rho and div v for sinusoidal fields, du/dt = -(P/rho) div v
for uniform rho and h, viscous heating only, Galilean invariance and a
viscosity that switches off in expansion.
"""
import math

import numpy as np
import pytest

from helpers import oracle_params, oracle_state
from paper_2007_03097_gb300 import inputs

EPS = np.finfo(np.float64).eps


def _random_state(orc, n_side=10, seed=7, kernel=1):
    w = inputs.lattice(n_side, jitter=0.3, kernel=kernel, fixed_h=False)
    rng = np.random.default_rng(seed)
    w.vx, w.vy, w.vz = rng.uniform(-1, 1, (3, w.n))
    w.u = rng.uniform(0.5, 1.5, w.n)
    p = oracle_params(orc, w, fixed_h=False)
    s = orc.evaluate(p, oracle_state(orc, w))
    return p, s


def test_momentum_and_energy_conservation(orc):
    p, s = _random_state(orc)
    assert s.extra["density_status"] == 0
    m = s.m
    tot = orc.totals(s)
    scale_f = np.sum(m * s.extra["S_a"])
    assert np.max(np.abs(tot["force"])) < 10 * EPS * scale_f
    vmag = np.sqrt(s.vx ** 2 + s.vy ** 2 + s.vz ** 2)
    scale_e = np.sum(m * (vmag * s.extra["S_a"] + s.extra["S_u"]))
    assert abs(tot["power"]) < 10 * EPS * scale_e
    # and the viscosity was active in this test
    p0 = oracle_params(orc, inputs.lattice(4), alpha=0.0, beta=0.0, kernel=p.kernel, eta=p.eta)
    f0 = orc.forces(p0, s.x, s.y, s.z, s.vx, s.vy, s.vz, s.m, s.h, s.rho, s.extra["P"], s.extra["c"])
    assert np.max(np.abs(f0.dudt - s.dudt)) > 1e-3 * np.max(np.abs(s.dudt))


def test_perfect_lattice_at_rest_has_no_force(orc):
    w = inputs.lattice(8, jitter=0.0, kernel=0, fixed_h=True)
    p = oracle_params(orc, w)
    s = orc.evaluate(p, oracle_state(orc, w))
    S = s.extra["S_a"]
    for a in (s.ax, s.ay, s.az):
        assert np.max(np.abs(a) / S) < 1e-13
    assert np.all(s.dudt == 0)
    # v = 0: the signal speed is c_a + c_b = 2c
    assert np.allclose(s.vsig, 2 * s.extra["c"], rtol=1e-15)


def _sine_lattice(orc, n_side, kernel=1):
    w = inputs.lattice(n_side, jitter=0.0, kernel=kernel, fixed_h=True)
    p = oracle_params(orc, w, alpha=0.0, beta=0.0)
    d = orc.density(p, w.x, w.y, w.z, w.m, w.h)
    return w, p, d


def _offset_sine_sum(orc, kernel, n_side, h, k):
    """F = sum over lattice offsets d of sin(k d_x) W'(|d|, h) d_x / |d|, the one
    lattice constant that a sinusoidal field in x reduces the pair sums to."""
    dx = 1.0 / n_side
    o = np.arange(-3, 4)
    ox, oy, oz = np.meshgrid(o, o, o, indexing="ij")
    d = np.stack([ox.ravel(), oy.ravel(), oz.ravel()]).astype(np.float64) * dx
    r = np.sqrt((d * d).sum(axis=0))
    keep = (r > 0) & (r < 2 * h)
    _, dW, _ = orc.kernel(kernel, r[keep], h)
    return float(np.sum(np.sin(k * d[0, keep]) * dW * d[0, keep] / r[keep]))


def test_pressure_gradient_on_lattice(orc):
    """u = u0 (1 + A sin kx) at uniform rho.  On a perfect lattice the pair
    sum of Eq. 6 reduces to a_x = (m/rho)(gamma-1) u0 A cos(kx) F, and
    (m/rho) F -> -k in the continuum: a = -grad P / rho."""
    n_side = 24
    w, p, d = _sine_lattice(orc, n_side)
    A, u0, k = 0.01, 1.0, 2 * math.pi
    u = u0 * (1 + A * np.sin(k * w.x))
    P, c = orc.eos(p.gamma, d.rho, u)
    t = np.arange(0, w.n, 97)
    f = orc.forces(p, w.x, w.y, w.z, w.vx, w.vy, w.vz, w.m, d.h, d.rho, P, c, targets=t)
    F = _offset_sine_sum(orc, p.kernel, n_side, w.h[0], k)
    m_rho = w.m[0] / d.rho[0]
    exact = m_rho * (p.gamma - 1) * u0 * A * np.cos(k * w.x[t]) * F
    amp = (p.gamma - 1) * u0 * A * k
    assert np.max(np.abs(f.ax[t] - exact)) < 1e-11 * amp
    assert abs(m_rho * F / -k - 1) < 0.06              # smoothing error (kh)^2 ~ 0.1
    assert np.max(np.abs(f.ay[t])) < 1e-10 * amp and np.max(np.abs(f.az[t])) < 1e-10 * amp


def test_divergence_and_compressional_heating(orc):
    """v_x = A sin kx: div v = -(m/rho) A cos(kx) F on the lattice (-> k A cos kx),
    and at uniform rho and h, du/dt = -(P/rho) div v (same pair sum in Eq. 5)."""
    n_side = 24
    w, p, d = _sine_lattice(orc, n_side)
    A, k = 0.05, 2 * math.pi
    vx = A * np.sin(k * w.x)
    P, c = orc.eos(p.gamma, d.rho, w.u)
    t = np.arange(0, w.n, 89)
    f = orc.forces(p, w.x, w.y, w.z, vx, w.vy, w.vz, w.m, d.h, d.rho, P, c, targets=t)
    F = _offset_sine_sum(orc, p.kernel, n_side, w.h[0], k)
    exact = -(w.m[0] / d.rho[0]) * A * np.cos(k * w.x[t]) * F
    assert np.max(np.abs(f.divv[t] - exact)) < 1e-11 * k * A
    assert np.max(np.abs(f.divv[t] - k * A * np.cos(k * w.x[t]))) < 0.06 * k * A
    ref = -(P[t] / d.rho[t]) * f.divv[t]
    assert np.max(np.abs(f.dudt[t] - ref)) < 1e-12 * np.max(np.abs(ref))


def test_viscosity_only_heats(orc):
    w = inputs.lattice(8, jitter=0.3, kernel=1, fixed_h=False)
    rng = np.random.default_rng(3)
    w.vx, w.vy, w.vz = rng.uniform(-1, 1, (3, w.n))
    w.u = np.full(w.n, 1e-14)
    p = oracle_params(orc, w)
    s = orc.evaluate(p, oracle_state(orc, w))
    assert np.min(s.dudt) > -1e-10 * np.max(s.dudt)
    assert np.max(s.dudt) > 0


def test_galilean_invariance(orc):
    p, s = _random_state(orc, n_side=8)
    P, c = s.extra["P"], s.extra["c"]
    f1 = orc.forces(p, s.x, s.y, s.z, s.vx, s.vy, s.vz, s.m, s.h, s.rho, P, c)
    f2 = orc.forces(p, s.x, s.y, s.z, s.vx + 3.0, s.vy - 1.0, s.vz + 0.5, s.m, s.h, s.rho, P, c)
    S = f1.S_a
    for a, b in ((f1.ax, f2.ax), (f1.ay, f2.ay), (f1.az, f2.az)):
        assert np.max(np.abs(a - b) / S) < 1e-12
    assert np.max(np.abs(f1.dudt - f2.dudt) / np.maximum(f1.S_u, 1e-300)) < 1e-11


def test_viscosity_off_in_expansion(orc):
    rng = np.random.default_rng(5)
    n = 300
    x, y, z = rng.normal(size=(3, n)) * 0.2
    vx, vy, vz = 0.1 * x, 0.1 * y, 0.1 * z
    m = np.full(n, 1.0 / n)
    p = orc.Params(kernel=1, periodic=False, h_max=20.0, eta=1.2)
    d = orc.density(p, x, y, z, m, np.full(n, 0.1))
    P, c = orc.eos(p.gamma, d.rho, np.full(n, 1.0))
    f1 = orc.forces(p, x, y, z, vx, vy, vz, m, d.h, d.rho, P, c)
    p0 = orc.Params(kernel=1, periodic=False, h_max=20.0, eta=1.2, alpha=0.0, beta=0.0)
    f0 = orc.forces(p0, x, y, z, vx, vy, vz, m, d.h, d.rho, P, c)
    assert np.array_equal(f1.ax, f0.ax) and np.array_equal(f1.dudt, f0.dudt)


def test_target_subset_matches_full(orc):
    p, s = _random_state(orc, n_side=6)
    P, c = s.extra["P"], s.extra["c"]
    t = np.array([0, 5, 77, 215])
    f = orc.forces(p, s.x, s.y, s.z, s.vx, s.vy, s.vz, s.m, s.h, s.rho, P, c, targets=t)
    assert np.array_equal(f.ax[t], s.ax[t]) and np.array_equal(f.dudt[t], s.dudt[t])
