"""Pins of the size of the oracle's artificial viscosity, sound speed and
signal speed (Eqs. 5-6 with the Monaghan 1992 viscosity that Sec. 2.2.1 cites
as the standard prescription; the ideal-gas equation of state of Sec. 2.1).

Two particles in open space, M4 kernel in 3D, with hand-picked rational
positions, smoothing lengths, velocities, densities and sound speeds, so that
every quantity of the pair is a rational number times 1/pi.  The expected
values are worked out below step by step in exact fractions (the
intermediate results are written next to each step), from the printed forms

    mu_ab = h_ab (v_ab . r_ab) / (r_ab^2 + eps h_ab^2),     h_ab = (h_a + h_b)/2
    Pi_ab = (-alpha cbar_ab mu_ab + beta mu_ab^2) / rhobar_ab   (v_ab . r_ab < 0)
    a_a   = -m_b (P_a/rho_a^2 + P_b/rho_b^2 + Pi_ab) grad_a W(r_ab, h_ab)
    du_a  =  m_b (P_a/rho_a^2 + Pi_ab/2) v_ab . grad_a W(r_ab, h_ab)
    vsig_a = c_a + c_b - 3 min(0, v_ab . r_ab / r_ab)
    P = (gamma - 1) rho u,   c^2 = gamma P / rho = gamma (gamma - 1) u

and the M4 kernel W = w(q) / (pi h^3), dW/dr = w'(q) / (pi h^4) with
w'(q) = -(3/4)(2 - q)^2 on 1 <= q < 2.  The numbers are chosen so that each
plausible misreading changes the result: rhobar = 5/2 (Pi over rhobar^2),
|mu| != 1 (beta mu instead of beta mu^2), h_a != h_ab (mu built with h_a),
c_a != c_b (cbar), gamma = 5/3 (c = sqrt(gamma u)), an approach term of
3 |v_ab . rhat| (coefficient 1 instead of 3), and the alpha and beta terms
are also checked one at a time.
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest

PI = math.pi

# the pair: a at the origin, b at distance r = 9/10; h_a = 1/2, h_b = 7/10
H_A, H_B = F(1, 2), F(7, 10)
H_AB = (H_A + H_B) / 2                       # 3/5
R = F(9, 10)
Q_AB = R / H_AB                              # 3/2
# M4: w'(3/2) = -(3/4) (1/2)^2 = -3/16;  h_ab^4 = 81/625
DWDR_AB = F(-3, 4) * (2 - Q_AB) ** 2 / H_AB ** 4   # -625/432, times 1/pi
M_A, M_B = F(1, 4), F(1, 4)
RHO_A, RHO_B = F(2), F(3)                    # rhobar = 5/2
C_A, C_B = F(2), F(1)                        # cbar = 3/2
EPS_V = F(1, 100)


def _pi_ab(vdotr, alpha, beta):
    """Monaghan's Pi_ab for the pair above, exact (Fraction)."""
    if vdotr >= 0:
        return F(0)
    mu = H_AB * vdotr / (R * R + EPS_V * H_AB * H_AB)
    cbar = (C_A + C_B) / 2
    rbar = (RHO_A + RHO_B) / 2
    return (-alpha * cbar * mu + beta * mu * mu) / rbar


def test_worked_numbers():
    """The hand-worked intermediate values quoted in the comments below."""
    assert H_AB == F(3, 5) and Q_AB == F(3, 2) and DWDR_AB == F(-625, 432)
    # head-on: v_ab = (1, 0, 0), r_ab = (-9/10, 0, 0): v.r = -9/10,
    # mu = (3/5)(-9/10) / (81/100 + 9/2500) = -75/113
    assert H_AB * F(-9, 10) / (R * R + EPS_V * H_AB * H_AB) == F(-75, 113)
    assert _pi_ab(F(-9, 10), 1, 0) == F(45, 113)          # -(3/2)(-75/113)/(5/2)
    assert _pi_ab(F(-9, 10), 0, 2) == F(4500, 12769)      # 2 (75/113)^2 / (5/2)
    assert _pi_ab(F(-9, 10), 1, 2) == F(9585, 12769)
    # oblique: r_ab = -(9/10)(3/5, 4/5, 0), v.r = -27/50, mu = -45/113
    assert _pi_ab(F(-27, 50), 1, 2) == F(27, 113) + F(1620, 12769)


def _run(orc, xb, vb, alpha, beta, P=(0.0, 0.0), gamma=5.0 / 3.0):
    x = np.array([0.0, xb[0]])
    y = np.array([0.0, xb[1]])
    z = np.array([0.0, xb[2]])
    vx = np.array([0.5, vb[0]])
    vy = np.array([0.0, vb[1]])
    vz = np.array([0.0, vb[2]])
    m = np.array([float(M_A), float(M_B)])
    h = np.array([float(H_A), float(H_B)])
    rho = np.array([float(RHO_A), float(RHO_B)])
    c = np.array([float(C_A), float(C_B)])
    p = orc.Params(kernel=orc.M4, periodic=False, alpha=alpha, beta=beta, eps_visc=0.01, gamma=gamma,
                   h_max=100.0)
    return orc.forces(p, x, y, z, vx, vy, vz, m, h, rho, np.array(P, dtype=float), c)


def _close(got, want_fraction, over_pi=True, tol=4e-15):
    want = float(want_fraction) / (PI if over_pi else 1.0)
    assert got == pytest.approx(want, rel=tol, abs=1e-300), (got, want)


@pytest.mark.parametrize("alpha,beta,pi_exact", [
    (1.0, 0.0, F(45, 113)),                  # the alpha (linear, bulk) term alone
    (0.0, 2.0, F(4500, 12769)),              # the beta mu^2 (von Neumann-Richtmyer) term alone
    (1.0, 2.0, F(9585, 12769)),              # both, as in every workload
])
def test_head_on_pair(orc, alpha, beta, pi_exact):
    """b at (9/10, 0, 0) moving at -1/2 towards a moving at +1/2; P = 0, so
    the viscosity alone accelerates and heats the pair."""
    f = _run(orc, (0.9, 0.0, 0.0), (-0.5, 0.0, 0.0), alpha, beta)
    # grad_a W_ab = dW/dr r_ab / r = (-625/432)(-1, 0, 0) / pi = (625/432, 0, 0) / pi
    g = -DWDR_AB
    # a_a = -m_b Pi grad_a W;  a_b = -a_a (pair antisymmetry)
    _close(f.ax[0], -M_B * pi_exact * g)
    _close(f.ax[1], M_A * pi_exact * g)
    assert f.ay[0] == 0.0 and f.az[0] == 0.0
    # du_a = m_b (Pi/2) v_ab . grad_a W, v_ab = (1, 0, 0); the same for b
    _close(f.dudt[0], M_B * pi_exact / 2 * g)
    _close(f.dudt[1], M_A * pi_exact / 2 * g)
    # vsig = c_a + c_b + 3 |v_ab . rhat| = 2 + 1 + 3 * 1
    _close(f.vsig[0], F(6), over_pi=False)
    _close(f.vsig[1], F(6), over_pi=False)


def test_head_on_pair_with_pressure(orc):
    """P_a = 1, P_b = 3/2 with rho_a = 2, rho_b = 3: P_a/rho_a^2 = 1/4,
    P_b/rho_b^2 = 1/6 enter the momentum equation, only P_a/rho_a^2 the
    energy equation (with Pi/2)."""
    f = _run(orc, (0.9, 0.0, 0.0), (-0.5, 0.0, 0.0), 1.0, 2.0, P=(1.0, 1.5))
    pi_ab = F(9585, 12769)
    g = -DWDR_AB
    _close(f.ax[0], -M_B * (F(1, 4) + F(1, 6) + pi_ab) * g)
    _close(f.dudt[0], M_B * (F(1, 4) + pi_ab / 2) * g)
    _close(f.dudt[1], M_A * (F(1, 6) + pi_ab / 2) * g)


def test_oblique_pair(orc):
    """b at (9/10)(3/5, 4/5, 0) = (27/50, 18/25, 0), v_ab = (1, 0, 0):
    v_ab . r_ab = -27/50, the force is central (along r_ab)."""
    f = _run(orc, (0.54, 0.72, 0.0), (-0.5, 0.0, 0.0), 1.0, 2.0)
    pi_ab = F(27, 113) + F(1620, 12769)            # 4671/12769
    # grad_a W = (-625/432)(-(3/5), -(4/5), 0) / pi = (125/144, 125/108, 0) / pi
    gx, gy = F(125, 144), F(125, 108)
    _close(f.ax[0], -M_B * pi_ab * gx)
    _close(f.ay[0], -M_B * pi_ab * gy)
    _close(f.dudt[0], M_B * pi_ab / 2 * gx)        # v_ab . grad W = gx
    # vsig = 3 + 3 (27/50)/(9/10) = 24/5
    _close(f.vsig[0], F(24, 5), over_pi=False)


def test_receding_pair_has_no_viscosity(orc):
    f = _run(orc, (0.9, 0.0, 0.0), (1.5, 0.0, 0.0), 1.0, 2.0)
    assert f.ax[0] == 0.0 and f.dudt[0] == 0.0
    _close(f.vsig[0], F(3), over_pi=False)          # c_a + c_b, no approach term


def test_div_v_of_the_pair(orc):
    """div v_a = -(1/rho_a) m_b v_ab . grad_a W(r_ab, h_a): q_a = 9/5,
    w'(9/5) = -3/100, h_a^4 = 1/16, so grad_a W = (12/25, 0, 0) / pi and
    div v_a = -(1/2)(1/4)(12/25)/pi = -3/(50 pi).  For b, q_b = 9/7,
    w'(9/7) = -75/196, h_b^4 = 2401/10000: div v_b = -15625/(117649 pi)."""
    f = _run(orc, (0.9, 0.0, 0.0), (-0.5, 0.0, 0.0), 1.0, 2.0)
    _close(f.divv[0], F(-3, 50))
    _close(f.divv[1], F(-15625, 117649))


def test_ideal_gas_eos(orc):
    """P = (gamma - 1) rho u and the adiabatic sound speed c^2 = gamma P / rho
    (textbook ideal gas): gamma = 5/3, rho = 2, u = 3/4 give P = 1 and
    c^2 = 5/6; on random states c^2 = gamma P / rho to rounding."""
    P, c = orc.eos(5.0 / 3.0, np.array([2.0]), np.array([0.75]))
    assert P[0] == pytest.approx(1.0, rel=4e-16)
    assert c[0] ** 2 == pytest.approx(5.0 / 6.0, rel=4e-16)
    rng = np.random.default_rng(11)
    for gamma in (5.0 / 3.0, 1.4, 2.0, 1.01):
        rho = rng.uniform(0.01, 10.0, 1000)
        u = rng.uniform(1e-3, 1e3, 1000)
        P, c = orc.eos(gamma, rho, u)
        assert np.allclose(P / (rho * u), gamma - 1.0, rtol=1e-15, atol=0)
        assert np.allclose(c * c, gamma * P / rho, rtol=1e-14, atol=0)
