"""Pins of the oracle's exact Riemann solution (the analytic curves of the
Sod shock tube, Sec. 3), checked against what the Euler equations fix rather
than against the solver's own iteration: the Rankine-Hugoniot jumps across
the shock at the returned shock speed, the isentrope and Riemann invariant
through the rarefaction fan and its characteristic xi = u - c, continuity of
p and u across the contact, closed forms for symmetric double rarefactions
and symmetric collisions, and a uniform state left alone.
"""
import math

import numpy as np
import pytest

from oracle import riemann

SOD_L, SOD_R, GAMMA = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4


def _energy(rho, u, p, g):
    return p / (g - 1.0) + 0.5 * rho * u * u


def test_shock_satisfies_rankine_hugoniot():
    S = riemann.shock_speed(SOD_L, SOD_R, GAMMA)
    ps, us = riemann.star_state(SOD_L, SOD_R, GAMMA)
    r, u, p = riemann.sample(SOD_L, SOD_R, GAMMA, np.array([S - 1e-9, S + 1e-9]))
    assert r[1] == SOD_R[0] and p[1] == SOD_R[2]          # ahead: the right state
    assert p[0] == pytest.approx(ps, rel=1e-15) and u[0] == pytest.approx(us, rel=1e-15)
    # fluxes in the shock frame: mass, momentum, energy
    w = u - S
    mass = r * w
    mom = r * w * w + p
    en = (_energy(r, u, p, GAMMA) + p) * u - S * _energy(r, u, p, GAMMA)
    assert abs(mass[0] - mass[1]) < 1e-13 * abs(mass[1])
    assert abs(mom[0] - mom[1]) < 1e-13 * abs(mom[1])
    assert abs(en[0] - en[1]) < 1e-13 * abs(en[1])


def test_rarefaction_fan_is_isentropic_and_characteristic():
    ps, us = riemann.star_state(SOD_L, SOD_R, GAMMA)
    rl, ul, pl = SOD_L
    cl = math.sqrt(GAMMA * pl / rl)
    cs = cl * (ps / pl) ** ((GAMMA - 1) / (2 * GAMMA))
    head, tail = ul - cl, us - cs
    xi = np.linspace(head, tail, 41)[1:-1]
    r, u, p = riemann.sample(SOD_L, SOD_R, GAMMA, xi)
    c = np.sqrt(GAMMA * p / r)
    assert np.max(np.abs(p / r ** GAMMA / (pl / rl ** GAMMA) - 1)) < 1e-13
    inv = u + 2 * c / (GAMMA - 1)
    assert np.max(np.abs(inv - (ul + 2 * cl / (GAMMA - 1)))) < 1e-13
    assert np.max(np.abs(u - c - xi)) < 1e-13
    assert np.all(np.diff(p) < 0) and np.all(np.diff(u) > 0)


def test_contact_carries_pressure_and_velocity():
    ps, us = riemann.star_state(SOD_L, SOD_R, GAMMA)
    r, u, p = riemann.sample(SOD_L, SOD_R, GAMMA, np.array([us - 1e-9, us + 1e-9]))
    assert p[0] == p[1] == ps and u[0] == u[1] == us
    assert r[0] > r[1]                                    # the density jumps down across it
    # the star-left density lies on the left isentrope
    assert r[0] == pytest.approx(SOD_L[0] * (ps / SOD_L[2]) ** (1 / GAMMA), rel=1e-14)


@pytest.mark.parametrize("a", [0.2, 1.0])
def test_symmetric_double_rarefaction_closed_form(a):
    g, rho, p0 = 5.0 / 3.0, 1.0, 0.4
    c0 = math.sqrt(g * p0 / rho)
    ps, us = riemann.star_state((rho, -a, p0), (rho, a, p0), g)
    assert abs(us) < 1e-15
    exact = p0 * ((c0 - 0.5 * (g - 1) * a) / c0) ** (2 * g / (g - 1))
    assert ps == pytest.approx(exact, rel=1e-13)


@pytest.mark.parametrize("a", [0.3, 2.0])
def test_symmetric_collision_closed_form(a):
    g, rho, p0 = 1.4, 1.0, 1.0
    ps, us = riemann.star_state((rho, a, p0), (rho, -a, p0), g)
    A = 2.0 / ((g + 1) * rho)
    B = p0 * (g - 1) / (g + 1)
    # (p - p0)^2 A = a^2 (p + B), the root above p0
    qa, qb, qc = A, -(2 * A * p0 + a * a), A * p0 * p0 - a * a * B
    exact = (-qb + math.sqrt(qb * qb - 4 * qa * qc)) / (2 * qa)
    assert abs(us) < 1e-14
    assert ps == pytest.approx(exact, rel=1e-13)


def test_uniform_state_stays():
    st = (0.7, 0.3, 2.0)
    ps, us = riemann.star_state(st, st, 1.4)
    assert ps == pytest.approx(2.0, rel=1e-15) and us == pytest.approx(0.3, rel=1e-15)
    r, u, p = riemann.sample(st, st, 1.4, np.linspace(-3, 3, 13))
    assert np.allclose(r, 0.7, rtol=1e-14) and np.allclose(u, 0.3, rtol=1e-14) and np.allclose(p, 2.0, rtol=1e-14)


def test_sod_star_region_textbook_values():
    """The star-region values of the Sod problem as printed to five decimals
    in Toro's textbook (tests/golden/sod_star_region.txt)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sod_star_region.txt")
    ref = {}
    with open(path) as f:
        for line in f:
            t = line.split()
            if t and not t[0].startswith("#"):
                ref[t[0]] = float(t[1])
    p, u = riemann.star_state(SOD_L, SOD_R, GAMMA)
    rl = riemann.sample(SOD_L, SOD_R, GAMMA, np.array([u - 1e-9]))[0][0]
    rr = riemann.sample(SOD_L, SOD_R, GAMMA, np.array([u + 1e-9]))[0][0]
    got = {"p_star": p, "u_star": u, "rho_star_L": rl, "rho_star_R": rr}
    for k, v in ref.items():
        assert abs(got[k] - v) <= 5e-6, (k, got[k], v)
