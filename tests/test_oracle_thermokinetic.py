"""Pins of the oracle's thermokinetic energy equation (Sec. 2.1, Eq. thermo):
de_a/dt of the specific total energy e = u + v^2/2.

Independent checks: at the semi-discrete level the pair sum equals
du_a/dt + v_a . dv_a/dt of Eqs. 5-6 for every particle (expanding
v_ab = v_a - v_b in Eq. 5 gives the thermokinetic terms); the pair terms are
antisymmetric, so sum_a m_a de_a/dt vanishes to roundoff; particles at rest
have no energy rate; and the leapfrog that advances e conserves the total
energy to roundoff while the one advancing u has an O(dt^2) error.
"""
import numpy as np

from helpers import oracle_params, oracle_state
from paper_2007_03097_gb300 import inputs

EPS = np.finfo(np.float64).eps


def _state(orc, n_side=8, seed=3, vamp=1.0, alpha=1.0, beta=2.0):
    w = inputs.lattice(n_side, jitter=0.3, kernel=1, fixed_h=False)
    rng = np.random.default_rng(seed)
    w.vx, w.vy, w.vz = vamp * rng.uniform(-1, 1, (3, w.n))
    w.u = rng.uniform(0.5, 1.5, w.n)
    p = oracle_params(orc, w, fixed_h=False, alpha=alpha, beta=beta)
    s = orc.evaluate(p, oracle_state(orc, w), thermokinetic=True)
    return p, s


def test_equals_du_plus_v_dot_a(orc):
    p, s = _state(orc)
    assert s.extra["density_status"] == 0
    lhs = s.dedt
    rhs = s.dudt + (s.vx * s.ax + s.vy * s.ay + s.vz * s.az)
    vmag = np.sqrt(s.vx ** 2 + s.vy ** 2 + s.vz ** 2)
    scale = s.extra["S_e"] + s.extra["S_u"] + vmag * s.extra["S_a"]
    assert np.max(np.abs(lhs - rhs) / scale) < 1e-13
    assert np.max(np.abs(lhs)) > 1e-3 * np.max(scale)           # not trivially zero


def test_total_energy_rate_vanishes(orc):
    p, s = _state(orc, seed=5)
    total = np.sum(s.m * s.dedt)
    assert abs(total) < 20 * EPS * np.sum(s.m * s.extra["S_e"])
    assert np.max(np.abs(s.dedt)) > 0.0


def test_particles_at_rest_have_no_energy_rate(orc):
    p, s = _state(orc, vamp=0.0)
    assert np.all(s.dedt == 0.0)


def test_leapfrog_conserves_total_energy(orc):
    p, s0 = _state(orc, n_side=6, seed=9, vamp=0.5)
    E0 = orc.totals(s0)["energy"]
    dt = 0.5 * orc.cfl_dt(s0)
    s_e, s_u = s0.copy(), s0.copy()
    for _ in range(6):
        s_e = orc.kdk_step_thermokinetic(p, s_e, dt)
        s_u = orc.kdk_step(p, s_u, dt)
    err_e = abs(orc.totals(s_e)["energy"] - E0)
    err_u = abs(orc.totals(s_u)["energy"] - E0)
    assert err_e < 1e-13 * abs(E0)
    assert err_u > 100 * err_e
