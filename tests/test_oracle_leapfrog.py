"""Pins of the oracle's kick-drift-kick leapfrog (the paper names no
integrator; the method needs one to advance Eqs. 5-6).

Independent checks: second-order energy error (halving dt cuts the energy
error about four-fold), momentum conserved to roundoff over many steps, and
a free-streaming check (no pressure, no viscosity: x advances by v t exactly).
"""
import numpy as np

from helpers import oracle_params, oracle_state
from paper_2007_03097_gb300 import inputs


def _small(orc, alpha=0.0, beta=0.0, vamp=0.3, n_side=6):
    w = inputs.lattice(n_side, jitter=0.2, kernel=1, fixed_h=False)
    rng = np.random.default_rng(11)
    w.vx, w.vy, w.vz = vamp * rng.uniform(-1, 1, (3, w.n))
    p = oracle_params(orc, w, alpha=alpha, beta=beta)
    s = orc.evaluate(p, oracle_state(orc, w))
    return p, s


def _run(orc, p, s, dt, nsteps):
    for _ in range(nsteps):
        s = orc.kdk_step(p, s, dt)
    return s


def test_energy_error_is_second_order(orc):
    p, s0 = _small(orc)
    E0 = orc.totals(s0)["energy"]
    T = 0.02
    errs = []
    for nst in (4, 8):
        s = _run(orc, p, s0.copy(), T / nst, nst)
        errs.append(abs(orc.totals(s)["energy"] - E0))
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.5, ratio


def test_momentum_conserved_with_viscosity(orc):
    p, s = _small(orc, alpha=1.0, beta=2.0, vamp=1.0)
    P0 = orc.totals(s)["momentum"]
    s = _run(orc, p, s, 2e-3, 5)
    P1 = orc.totals(s)["momentum"]
    scale = np.sum(s.m * np.sqrt(s.vx ** 2 + s.vy ** 2 + s.vz ** 2))
    assert np.max(np.abs(P1 - P0)) < 1e-13 * scale


def test_free_streaming(orc):
    """u = 0 and no viscosity: no force, so x(t) = x0 + v t (periodic wrap)."""
    w = inputs.lattice(5, jitter=0.2, kernel=1, fixed_h=False, u0=0.0)
    rng = np.random.default_rng(2)
    w.vx, w.vy, w.vz = rng.uniform(-1, 1, (3, w.n))
    p = oracle_params(orc, w, alpha=0.0, beta=0.0)
    s = orc.evaluate(p, oracle_state(orc, w))
    dt, nst = 0.01, 3
    s1 = _run(orc, p, s.copy(), dt, nst)
    for x0, v, x1 in ((s.x, s.vx, s1.x), (s.y, s.vy, s1.y), (s.z, s.vz, s1.z)):
        ref = np.mod(x0 + v * dt * nst, 1.0)
        d = np.abs(x1 - ref)
        assert np.max(np.minimum(d, 1 - d)) < 1e-14
    assert np.all(s1.u == 0)
