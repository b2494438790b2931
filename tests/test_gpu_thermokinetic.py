"""GPU parity of the thermokinetic formulation (Sec. 2.1, Eq. thermo) against
the oracle: the force pass's de/dt, a kick-drift-kick run that advances the
specific total energy, and the total energy it conserves to roundoff."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import need_gpu, to_oracle_params
from helpers import oracle_state
from paper_2007_03097_gb300 import inputs

pytestmark = pytest.mark.gpu


def _moving_gas(n_side, seed=21, vamp=0.3):
    """Jittered periodic lattice of warm gas (u ~ 1) in random motion,
    Wendland C2, variable h: the thermokinetic form recovers u = e - v^2/2, so
    the kinetic energy must not dwarf the thermal one."""
    w = inputs.lattice(n_side, jitter=0.3, kernel=1, fixed_h=False)
    rng = np.random.default_rng(seed)
    w.vx, w.vy, w.vz = vamp * rng.uniform(-1, 1, (3, w.n))
    w.u = rng.uniform(0.5, 1.5, w.n)
    w.params["energy"] = 1
    return w


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-4)])
def test_energy_rate_matches_oracle(precision, tol):
    B = need_gpu()
    w = _moving_gas(14)
    w.params["precision"] = precision
    fp64 = precision == "fp64"
    ctx = B.Context(w.params, w.n)
    p = B.Particles.from_workload(w, fp64=fp64)
    B.sph_build_tree(ctx, p)
    B.sph_density(ctx, p)
    st = B.sph_forces(ctx, p)
    g = p.numpy()
    op = to_oracle_params(oracle, w.params)
    f64 = lambda k: np.asarray(g[k], dtype=np.float64)
    P, c = oracle.eos(op.gamma, f64("rho"), f64("u"))
    dedt, se = oracle.energy_rate(op, g["x"], g["y"], g["z"], f64("vx"), f64("vy"), f64("vz"), f64("m"),
                                  f64("h"), f64("rho"), P, c)
    err = np.max(np.abs(f64("dudt") - dedt) / np.maximum(se, 1e-300))
    assert err < tol, err
    assert st["interactions"] > 0


def test_steps_match_oracle_and_conserve_energy():
    w = _moving_gas(12)
    B = need_gpu()
    ctx = B.Context(w.params, w.n)
    p = B.Particles.from_workload(w, fp64=True)
    B.sph_build_tree(ctx, p)
    B.sph_density(ctx, p)
    B.sph_forces(ctx, p)
    op = to_oracle_params(oracle, w.params)
    s = oracle.evaluate(op, oracle_state(oracle, w), thermokinetic=True)
    E0 = oracle.totals(s)["energy"]
    dt = 0.5 * oracle.cfl_dt(s)
    worst = {}
    for k in range(12):
        st = B.sph_step(ctx, p, dt)
        s = oracle.kdk_step_thermokinetic(op, s, dt)
        assert np.all(np.isfinite(s.u)) and np.all(s.u > 0)
        g = p.in_original_order()
        for f in ("vx", "vy", "vz", "u", "h", "rho", "dudt"):
            ref = getattr(s, "dedt" if f == "dudt" else f)
            e = np.max(np.abs(g[f] - ref)) / max(np.max(np.abs(ref)), 1e-300)
            worst[f] = max(worst.get(f, 0.0), e)
    assert max(worst.values()) < 1e-10, worst
    # total energy of the GPU run: conserved to roundoff (the step's FP64 totals)
    assert abs(st["energy"] - E0) < 1e-12 * abs(E0)
    assert abs(st["power"]) < 1e-10 * np.sum(s.m * s.extra["S_e"])
