"""GPU parity of the kick-drift-kick step against the oracle: a Sedov blast
(reduced to 16^3 particles so the brute-force oracle keeps up) advanced 50
steps with the fixed step of the workload, FP64, compared field by field;
conserved totals; the CFL step."""
import numpy as np
import pytest

import oracle
from gpu_helpers import need_gpu, to_oracle_params
from helpers import oracle_state
from paper_2007_03097_gb300 import inputs

pytestmark = pytest.mark.gpu


def _gpu_init(w, fp64=True):
    B = need_gpu()
    ctx = B.Context(w.params, w.n)
    p = B.Particles.from_workload(w, fp64=fp64)
    B.sph_build_tree(ctx, p)
    B.sph_density(ctx, p)
    B.sph_forces(ctx, p)
    return B, ctx, p


def _scaled_err(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def test_sedov_50_steps_fp64():
    w = inputs.sedov(16, steps=50)
    B, ctx, p = _gpu_init(w)
    op = to_oracle_params(oracle, w.params)
    s = oracle.evaluate(op, oracle_state(oracle, w))
    worst = {}
    for k in range(w.steps):
        st = B.sph_step(ctx, p, w.dt)
        s = oracle.kdk_step(op, s, w.dt)
        if k % 10 == 9 or k == w.steps - 1:
            g = p.in_original_order()
            for f in ("x", "y", "z"):
                d = np.abs(g[f] - getattr(s, f))
                d = np.minimum(d, 1.0 - d)                      # periodic
                worst[f] = max(worst.get(f, 0), np.max(d) / np.max(s.h))
            for f in ("vx", "vy", "vz", "u", "h", "rho", "ax", "dudt"):
                worst[f] = max(worst.get(f, 0), _scaled_err(g[f], getattr(s, f)))
    assert max(worst.values()) < 1e-10, worst
    assert st["density"]["n_unconverged"] == 0


def test_step_conserves_momentum_and_energy_rate():
    w = inputs.sedov(12)
    B, ctx, p = _gpu_init(w)
    P0 = B.sph_totals(ctx, p)[:3]
    for _ in range(5):
        st = B.sph_step(ctx, p, w.dt)
    mom = np.array(st["momentum"])
    g = p.numpy()
    scale = np.sum(g["m"] * np.sqrt(g["vx"] ** 2 + g["vy"] ** 2 + g["vz"] ** 2))
    assert np.max(np.abs(mom - P0)) < 1e-12 * scale
    fscale = np.sum(g["m"] * np.sqrt(g["ax"] ** 2 + g["ay"] ** 2 + g["az"] ** 2))
    assert np.max(np.abs(st["force"])) < 1e-12 * fscale
    pscale = np.sum(g["m"] * (np.sqrt(g["vx"] ** 2 + g["vy"] ** 2 + g["vz"] ** 2) *
                              np.sqrt(g["ax"] ** 2 + g["ay"] ** 2 + g["az"] ** 2) + np.abs(g["dudt"])))
    assert abs(st["power"]) < 1e-11 * pscale


def test_cfl_step_matches_definition():
    w = inputs.sedov(12)
    B, ctx, p = _gpu_init(w)
    st = B.sph_step(ctx, p, w.dt)
    g = p.numpy()
    assert st["dt_next"] == pytest.approx(w.params["cfl"] * np.min(g["h"] / g["vsig"]), rel=1e-14)
    st2 = B.sph_step(ctx, p, 0.0)                  # dt <= 0: use the stored CFL step
    assert st2["dt"] == st["dt_next"]


def test_mixed_step_runs_and_conserves_momentum():
    w = inputs.polytrope(20000, seed=3, precision="mixed")
    B, ctx, p = _gpu_init(w, fp64=False)
    P0 = B.sph_totals(ctx, p)[:3]
    for _ in range(3):
        st = B.sph_step(ctx, p, 1e-3)
    g = p.numpy()
    scale = np.sum(g["m"] * np.sqrt(g["vx"] ** 2 + g["vy"] ** 2 + g["vz"] ** 2)) + 1e-300
    assert np.max(np.abs(np.array(st["momentum"]) - P0)) < 1e-5 * scale
    assert st["density"]["n_unconverged"] == 0
