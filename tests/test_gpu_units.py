"""FP64 mode in the paper's own units.  Sec. 3.2 runs its star in CGS (masses
near 10^33 g, lengths near 10^10 cm, specific energies near 10^15 erg/g).  The
double-float pair arithmetic of FP64 mode has the exponent range of FP32, so
the library changes length and mass units by exact powers of two before the
pair sums and back after them.  Here the config-1 lattice scaled to CGS
magnitudes is compared with the FP64 oracle in the same units: the fixed-h
evaluation to 1e-12 and, with star-like u and v, the variable-h evaluation to
1e-10; and the scaled run equals the unit-box run transformed back."""
import numpy as np
import pytest

import oracle
from gpu_helpers import need_gpu, to_oracle_params
from paper_2007_03097_gb300 import inputs

pytestmark = pytest.mark.gpu

LU, MU = 1e10, 2e33          # cm per code length, g per code mass


def _cgs(w, u_scale=1.0, v_scale=1.0):
    """The workload in CGS-sized units: lengths x LU, masses x MU, velocities
    x v_scale and specific energies x u_scale (the caller's choice)."""
    for k in ("x", "y", "z", "h"):
        setattr(w, k, getattr(w, k) * LU)
    w.m = w.m * MU
    for k in ("vx", "vy", "vz"):
        setattr(w, k, getattr(w, k) * v_scale)
    w.u = w.u * u_scale
    w.params = dict(w.params, box_lo=(0.0, 0.0, 0.0), box_hi=(LU, LU, LU),
                    h_min=w.params["h_min"] * LU, h_max=w.params["h_max"] * LU)
    return w


def _run(w):
    B = need_gpu()
    ctx = B.Context(w.params, w.n)
    p = B.Particles.from_workload(w, fp64=True)
    B.sph_build_tree(ctx, p)
    ds = B.sph_density(ctx, p)
    B.sph_forces(ctx, p)
    return B, ctx, p, ds


def _compare(w, tol):
    B, ctx, p, ds = _run(w)
    g = p.in_original_order()
    op = to_oracle_params(oracle, w.params)
    d = oracle.density(op, w.x, w.y, w.z, w.m, w.h)
    assert np.array_equal(g["nnb"], d.nnb)
    assert np.max(np.abs(g["h"] / d.h - 1)) < tol
    assert np.max(np.abs(g["rho"] / d.rho - 1)) < tol
    # omega is drho/dh at the last evaluated h: within |dh| < h_tol h of the
    # final h when the last step was taken to first order (variable h)
    tol_om = tol if w.params["fixed_h"] else 1e-5
    assert np.max(np.abs(g["omega"] - d.drho_dh)) < tol_om * np.abs(d.drho_dh).max()
    P, c = oracle.eos(op.gamma, d.rho, w.u)
    f = oracle.forces(op, w.x, w.y, w.z, w.vx, w.vy, w.vz, w.m, d.h, d.rho, P, c)
    for k in ("ax", "ay", "az"):
        assert np.all(np.isfinite(g[k]))
        assert np.max(np.abs(g[k] - getattr(f, k)) / f.S_a) < tol, k
    assert np.max(np.abs(g["dudt"] - f.dudt) / np.maximum(f.S_u, 1e-300)) < tol
    if np.abs(f.divv).max() > 0:
        assert np.max(np.abs(g["divv"] - f.divv)) < tol * np.abs(f.divv).max()
    assert np.max(np.abs(g["vsig"] / f.vsig - 1)) < tol
    return g


def test_cgs_lattice_fixed_h():
    """Config 1 (16^3 jittered lattice, M4, fixed h = 1.2 spacings, u = 1,
    v = 0) with lengths in cm (box 10^10 cm) and masses in g (2 10^33 g):
    one density and force evaluation to 1e-12 against the oracle in CGS."""
    _compare(_cgs(inputs.lattice(16)), 1e-12)


def test_cgs_lattice_variable_h_moving():
    """The same lattice with variable h (eta 1.2), star-like specific energy
    (10^15 erg/g) and random velocities of 3 10^7 cm/s, so that the
    viscosity acts: h-rho iteration and forces to 1e-10."""
    w = inputs.lattice(16, jitter=0.2, fixed_h=False)
    rng = np.random.default_rng(12)
    w.vx, w.vy, w.vz = rng.standard_normal((3, w.n))
    w.u = rng.uniform(0.5, 1.5, w.n)
    _compare(_cgs(w, u_scale=1e15, v_scale=3e7), 1e-10)


def test_cgs_run_is_the_unit_box_run_transformed():
    """Exact unit changes commute with the method: the CGS run's rho, a and
    du/dt are the unit-box run's times MU/LU^3, v^2/LU and v^3/LU (v = 3e7
    cm/s per code velocity, u in (3e7)^2), to 1e-10 (the h iterations of the
    two runs may stop one sweep apart)."""
    V = 3e7
    w0 = inputs.lattice(12, jitter=0.2, fixed_h=False)
    rng = np.random.default_rng(5)
    w0.vx, w0.vy, w0.vz = rng.standard_normal((3, w0.n))
    w0.u = rng.uniform(0.5, 1.5, w0.n)
    B, c0, p0, _ = _run(w0)
    g0 = p0.in_original_order()
    w1 = inputs.lattice(12, jitter=0.2, fixed_h=False)
    w1.vx, w1.vy, w1.vz, w1.u = w0.vx.copy(), w0.vy.copy(), w0.vz.copy(), w0.u.copy()
    B, c1, p1, _ = _run(_cgs(w1, u_scale=V * V, v_scale=V))
    g1 = p1.in_original_order()
    assert np.array_equal(g0["nnb"], g1["nnb"])
    assert np.max(np.abs(g1["h"] / (g0["h"] * LU) - 1)) < 1e-10
    assert np.max(np.abs(g1["rho"] / (g0["rho"] * MU / LU ** 3) - 1)) < 1e-10
    scale_a = np.abs(g0["ax"]).max()
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(g1[k] / (V * V / LU) - g0[k])) < 1e-10 * scale_a
    assert np.max(np.abs(g1["dudt"] / (V ** 3 / LU) - g0["dudt"])) < 1e-10 * np.abs(g0["dudt"]).max()
