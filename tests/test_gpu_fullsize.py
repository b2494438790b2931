"""Parity at the full workload sizes, on sampled targets the brute-force
oracle evaluates one by one against ALL sources:

* Sedov blast 64^3 (FP64): h, rho to 1e-10 and forces to 1e-10 of their
  scale after the initial evaluation and after leapfrog steps;
* n = 1 polytrope, 2^20 particles (FP32 pairs, FP64 positions): rho, h to
  1e-5, a and du/dt to 1e-4 of their scale, including the smallest- and
  largest-h particles;
* two colliding polytropes, 2 x 2^21 particles: learned-h and plain-h seeds
  converge to the same h within 2 h_tol;
* periodic turbulence box 256^3 (Wendland C4, mixed): sampled rho, h, a.

The oracle is seeded with the GPU's converged h, so it checks that h is the
fixed point of Eq. 9 for the GPU's positions (Newton from there takes one
step below tolerance) and evaluates rho, a from the definitions.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import need_gpu, to_oracle_params
from paper_2007_03097_gb300 import inputs

pytestmark = pytest.mark.gpu


def _targets(g, n_rand, n_ext, seed=0):
    rng = np.random.default_rng(seed)
    n = g["x"].size
    t = set(rng.choice(n, size=min(n_rand, n), replace=False).tolist())
    order = np.argsort(g["h"])
    t.update(order[:n_ext].tolist())
    t.update(order[-n_ext:].tolist())
    return np.array(sorted(t), dtype=np.int64)


def _check(op, g, t, tol_rho, tol_a, w_u=None):
    d = oracle.density(op, g["x"], g["y"], g["z"], g["m"], g["h"], targets=t)
    assert not (d.flags[t] & oracle.NOT_CONVERGED).any()
    err_h = np.max(np.abs(d.h[t] / g["h"][t] - 1))
    err_rho = np.max(np.abs(d.rho[t] / g["rho"][t] - 1))
    assert np.array_equal(d.nnb[t], g["nnb"][t]) or tol_rho > 1e-8
    # forces from the GPU's own state of every source particle
    f = oracle.forces(op, g["x"], g["y"], g["z"], g["vx"], g["vy"], g["vz"], g["m"], g["h"], g["rho"], g["P"],
                      g["c"], targets=t)
    err_a = max(np.max(np.abs(g[k][t] - getattr(f, k)[t]) / np.maximum(f.S_a[t], 1e-300)) for k in ("ax", "ay", "az"))
    err_u = np.max(np.abs(g["dudt"][t] - f.dudt[t]) / np.maximum(f.S_u[t], 1e-300))
    assert err_h < tol_rho and err_rho < tol_rho, (err_h, err_rho)
    assert err_a < tol_a and err_u < tol_a, (err_a, err_u)
    return err_rho, err_a


def test_sedov_64_fp64_sampled():
    B = need_gpu()
    w = inputs.sedov(64)
    ctx = B.Context(w.params, w.n)
    p = B.Particles.from_workload(w, fp64=True)
    B.sph_build_tree(ctx, p)
    B.sph_density(ctx, p)
    B.sph_forces(ctx, p)
    op = to_oracle_params(oracle, w.params)
    g = p.numpy()
    hot = np.nonzero(g["u"] > 1.0)[0]
    t = np.unique(np.concatenate([_targets(g, 400, 32), hot]))
    _check(op, g, t, 1e-10, 1e-10)
    for _ in range(5):
        B.sph_step(ctx, p, w.dt)
    # re-evaluate density and forces at the end state through the stand-alone calls
    B.sph_build_tree(ctx, p)
    B.sph_density(ctx, p)
    B.sph_forces(ctx, p)
    g = p.numpy()
    near = np.argsort((g["x"] - 0.5) ** 2 + (g["y"] - 0.5) ** 2 + (g["z"] - 0.5) ** 2)[:200]
    t = np.unique(np.concatenate([_targets(g, 300, 32, seed=1), near]))
    _check(op, g, t, 1e-10, 1e-10)


def test_polytrope_1M_mixed_sampled():
    B = need_gpu()
    w = inputs.polytrope(1 << 20, precision="mixed")
    ctx = B.Context(w.params, w.n)
    p = B.Particles.from_workload(w, fp64=False)
    B.sph_build_tree(ctx, p)
    st = B.sph_density(ctx, p)
    assert st["n_unconverged"] == 0
    B.sph_forces(ctx, p)
    g = p.numpy()
    op = to_oracle_params(oracle, w.params)
    t = _targets(g, 256, 64)
    _check(op, g, t, 1e-5, 1e-4)
    spread = g["h"].max() / g["h"].min()
    assert spread > 5.0          # the star's h range (reported by the bench/DESIGN)


def test_collision_learned_vs_plain_h():
    """Two 2^21-particle polytropes: the trained predictor's seed and the plain
    seed converge to the same h (2 h_tol), and the seeded run needs no more
    particle evaluations than the plain one."""
    B = need_gpu()
    w = inputs.collision(1 << 21, precision="mixed")
    params = dict(w.params, hnet_batch=32768, hnet_iters=30, hnet_lr=2e-3)
    ctx = B.Context(params, w.n)
    p = B.Particles.from_workload(w, fp64=False)
    B.sph_build_tree(ctx, p)
    B.sph_density(ctx, p)
    B.sph_forces(ctx, p)
    dt = 2e-3
    for _ in range(6):                                   # plain steps that also train the network
        B.sph_step(ctx, p, dt, use_hnet=B.SPH_HNET_TRAIN)
    ctx.set_params(dict(params, hnet_iters=1))
    snap = {f: getattr(p, f).clone() for f in ["x", "y", "z", "nnb", "id"] + B._FIELDS}
    s_plain = B.sph_step(ctx, p, dt)
    h_plain = p.in_original_order(["h"])["h"]
    for f, v in snap.items():
        getattr(p, f).copy_(v)
    s_learn = B.sph_step(ctx, p, dt, use_hnet=B.SPH_HNET_SEED)
    h_learn = p.in_original_order(["h"])["h"]
    assert s_learn["hnet_used"] == 1
    assert np.max(np.abs(h_learn / h_plain - 1)) < 2 * w.params["h_tol"]
    print("evaluations plain", s_plain["density"]["evaluations"], "learned", s_learn["density"]["evaluations"],
          "sweeps", s_plain["density"]["sweeps"], s_learn["density"]["sweeps"])
    assert s_learn["density"]["evaluations"] <= 1.02 * s_plain["density"]["evaluations"]


def test_turbulence_256_mixed_sampled():
    B = need_gpu()
    w = inputs.turbulence(256)
    ctx = B.Context(w.params, w.n)
    p = B.Particles.from_workload(w, fp64=False)
    B.sph_build_tree(ctx, p)
    st = B.sph_density(ctx, p)
    assert st["n_unconverged"] == 0
    B.sph_forces(ctx, p)
    g = p.numpy()
    op = to_oracle_params(oracle, w.params)
    t = _targets(g, 96, 16)
    _check(op, g, t, 1e-5, 1e-4)
    nb = g["nnb"].mean()
    assert 90 < nb < 110                                 # ~100 neighbours with eta = 1.43971
