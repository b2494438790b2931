"""Parity at the full workload sizes, on sampled targets the brute-force
oracle evaluates one by one against ALL sources:

* Sedov blast 64^3 (FP64): h, rho, a, du/dt, div v and v_sig to 1e-10 after
  the initial evaluation and after the workload's 50 leapfrog steps;
* n = 1 polytrope, 2^20 particles (FP32 pairs, FP64 positions): rho, h to
  1e-5, a and du/dt to 1e-4 of their scale, div v and v_sig, including the
  smallest- and largest-h particles;
* two colliding polytropes, 2 x 2^21 particles, after steps seeded by the
  frozen h-predictor (trained on the plain solver's lattice and Sedov runs):
  the same tolerances, and learned-h and plain-h seeds converge to the same h
  within 2 h_tol with fewer density evaluations;
* periodic turbulence box 256^3 (Wendland C4, mixed): sampled rho, h, a.

The oracle is seeded with the GPU's converged h, so it checks that h is the
fixed point of Eq. 9 for the GPU's positions (Newton from there takes one
step below tolerance) and evaluates rho, a from the definitions.  Neighbour
counts must match exactly in FP64; in mixed precision every count that
differs must be explained by pairs within a relative 1e-5 of the support
radius (the FP32 and FP64 decisions may differ there), and the margins of
those pairs are printed.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import need_gpu, to_oracle_params
from paper_2007_03097_gb300 import inputs

pytestmark = pytest.mark.gpu

EDGE = 1e-5          # relative band of r^2 around a threshold where FP32 and FP64 decisions may differ


def _targets(g, n_rand, n_ext, seed=0):
    rng = np.random.default_rng(seed)
    n = g["x"].size
    t = set(rng.choice(n, size=min(n_rand, n), replace=False).tolist())
    order = np.argsort(g["h"])
    t.update(order[:n_ext].tolist())
    t.update(order[-n_ext:].tolist())
    return np.array(sorted(t), dtype=np.int64)


def _sep(op, d, axis):
    if op.periodic:
        L = op.box_hi[axis] - op.box_lo[axis]
        d = np.where(d > 0.5 * L, d - L, d)
        d = np.where(d < -0.5 * L, d + L, d)
    return d


def _edge_margins(op, g, a, kind):
    """Relative distances |r^2/thr - 1| of a's pairs near a threshold, FP64:
    kind "d" thr = 4 h_a^2, kind "f" thr = (h_a + h_b)^2."""
    dx = _sep(op, g["x"][a] - g["x"], 0)
    dy = _sep(op, g["y"][a] - g["y"], 1)
    dz = _sep(op, g["z"][a] - g["z"], 2)
    r2 = (dx * dx + dy * dy) + dz * dz
    thr = 4.0 * g["h"][a] ** 2 if kind == "d" else (g["h"][a] + g["h"]) ** 2
    rel = np.abs(r2 / thr - 1.0)
    rel[a] = np.inf
    return np.sort(rel[rel < EDGE])


def _check(op, g, t, tol_rho, tol_a, exact_sets):
    d = oracle.density(op, g["x"], g["y"], g["z"], g["m"], g["h"], targets=t)
    assert not (d.flags[t] & oracle.NOT_CONVERGED).any()
    err_h = np.max(np.abs(d.h[t] / g["h"][t] - 1))
    err_rho = np.max(np.abs(d.rho[t] / g["rho"][t] - 1))
    # neighbour counts: exact, or differing only through knife-edge pairs
    diff = np.nonzero(d.nnb[t] != g["nnb"][t])[0]
    if exact_sets:
        assert diff.size == 0, t[diff]
    for k in diff:
        a = t[k]
        m = _edge_margins(op, g, a, "d")
        print(f"nnb of {a}: GPU {g['nnb'][a]} oracle {d.nnb[a]}, knife-edge margins {m}")
        assert abs(int(d.nnb[a]) - int(g["nnb"][a])) <= m.size
    # forces from the GPU's own state of every source particle
    f = oracle.forces(op, g["x"], g["y"], g["z"], g["vx"], g["vy"], g["vz"], g["m"], g["h"], g["rho"], g["P"],
                      g["c"], targets=t)
    err_a = max(np.max(np.abs(g[k][t] - getattr(f, k)[t]) / np.maximum(f.S_a[t], 1e-300)) for k in ("ax", "ay", "az"))
    err_u = np.max(np.abs(g["dudt"][t] - f.dudt[t]) / np.maximum(f.S_u[t], 1e-300))
    assert err_h < tol_rho and err_rho < tol_rho, (err_h, err_rho)
    assert err_a < tol_a and err_u < tol_a, (err_a, err_u)
    # div v against the largest |div v| of the sample; v_sig relative, where a
    # knife-edge force pair may change which pair gives the maximum in FP32
    err_dv = np.max(np.abs(g["divv"][t] - f.divv[t])) / max(np.max(np.abs(f.divv[t])), 1e-300)
    assert err_dv < tol_a, err_dv
    rel_vs = np.abs(g["vsig"][t] / f.vsig[t] - 1)
    for k in np.nonzero(rel_vs > tol_rho)[0]:
        a = t[k]
        m = _edge_margins(op, g, a, "f")
        print(f"vsig of {a}: rel err {rel_vs[k]:.2e}, knife-edge force-pair margins {m}")
        assert not exact_sets and m.size > 0
    return err_rho, err_a


def test_sedov_64_fp64_sampled():
    """Config 2 at its full size: the initial evaluation and the state after
    the workload's 50 leapfrog steps (fixed dt)."""
    B = need_gpu()
    w = inputs.sedov(64)
    assert w.steps == 50
    ctx = B.Context(w.params, w.n)
    p = B.Particles.from_workload(w, fp64=True)
    B.sph_build_tree(ctx, p)
    B.sph_density(ctx, p)
    B.sph_forces(ctx, p)
    op = to_oracle_params(oracle, w.params)
    g = p.numpy()
    hot = np.nonzero(g["u"] > 1.0)[0]
    t = np.unique(np.concatenate([_targets(g, 400, 32), hot]))
    _check(op, g, t, 1e-10, 1e-10, exact_sets=True)
    for _ in range(w.steps):
        st = B.sph_step(ctx, p, w.dt)
    assert st["density"]["n_unconverged"] == 0
    # re-evaluate density and forces at the end state through the stand-alone calls
    B.sph_build_tree(ctx, p)
    B.sph_density(ctx, p)
    B.sph_forces(ctx, p)
    g = p.numpy()
    r2 = (g["x"] - 0.5) ** 2 + (g["y"] - 0.5) ** 2 + (g["z"] - 0.5) ** 2
    near = np.argsort(r2)[:200]
    shock = np.argsort(np.abs(np.sqrt(r2) - np.sqrt(r2[np.argmax(g["rho"])])))[:100]   # around the density peak
    t = np.unique(np.concatenate([_targets(g, 300, 32, seed=1), near, shock]))
    _check(op, g, t, 1e-10, 1e-10, exact_sets=True)
    assert np.max(g["rho"]) > 1.5                        # the blast has formed a shell


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
    _check(op, g, t, 1e-5, 1e-4, exact_sets=False)
    spread = g["h"].max() / g["h"].min()
    assert spread > 5.0          # the star's h range (reported by the bench/DESIGN)


@pytest.fixture(scope="module")
def protocol_theta():
    """The h-predictor trained by the protocol (200 plain steps each of the
    16^3 lattice with variable h and the 64^3 Sedov blast), then frozen."""
    need_gpu()
    from paper_2007_03097_gb300 import hnet_protocol
    theta, _ = hnet_protocol.train(steps=200)
    return theta


def test_collision_learned_steps_sampled(protocol_theta):
    """Config 4: two 2^21-particle polytropes.  After three steps seeded by
    the frozen network, the state is checked against the oracle on sampled
    targets (rho, h to 1e-5; a, du/dt to 1e-4).  From the same state a
    learned step and a plain step converge to the same h within 2 h_tol, and
    the learned step needs at least 5 % fewer density evaluations."""
    B = need_gpu()
    w = inputs.collision(1 << 21, precision="mixed")
    ctx = B.Context(dict(w.params, hnet_iters=1), w.n)
    p = B.Particles.from_workload(w, fp64=False)
    B.sph_build_tree(ctx, p)
    B.sph_density(ctx, p)
    B.sph_forces(ctx, p)
    B.sph_hnet_set_weights(ctx, protocol_theta)
    dt = 2e-3
    for _ in range(3):
        st = B.sph_step(ctx, p, dt, use_hnet=B.SPH_HNET_SEED)
        assert st["hnet_used"] == 1
    snap = {f: getattr(p, f).clone() for f in ["x", "y", "z", "nnb", "id"] + B._FIELDS}
    s_plain = B.sph_step(ctx, p, dt)
    h_plain = p.in_original_order(["h"])["h"]
    for f, v in snap.items():
        getattr(p, f).copy_(v)
    s_learn = B.sph_step(ctx, p, dt, use_hnet=B.SPH_HNET_SEED)
    h_learn = p.in_original_order(["h"])["h"]
    ev_p, ev_l = s_plain["density"]["evaluations"], s_learn["density"]["evaluations"]
    print("evaluations plain", ev_p, "learned", ev_l, "ratio", ev_l / ev_p, "fallbacks", s_learn["hnet_fallback"])
    assert np.max(np.abs(h_learn / h_plain - 1)) < 2 * w.params["h_tol"]
    assert ev_l < 0.95 * ev_p
    # the learned step's end state against the oracle
    B.sph_build_tree(ctx, p)
    B.sph_density(ctx, p)
    B.sph_forces(ctx, p)
    g = p.numpy()
    op = to_oracle_params(oracle, w.params)
    contact = np.argsort(np.abs(g["x"]))[:64]            # where the stars meet
    t = np.unique(np.concatenate([_targets(g, 160, 32, seed=3), contact]))
    _check(op, g, t, 1e-5, 1e-4, exact_sets=False)


def test_turbulence_learned_vs_plain_evaluations(protocol_theta):
    """Turbulence box (128^3, the headline workload's particles per volume at
    an eighth of the size): seeded by the frozen network, a step converges to
    the plain step's h within 2 h_tol with at least 20 % fewer density
    evaluations."""
    B = need_gpu()
    w = inputs.turbulence(128)
    ctx = B.Context(dict(w.params, hnet_iters=1), w.n)
    p = B.Particles.from_workload(w, fp64=False)
    B.sph_build_tree(ctx, p)
    B.sph_density(ctx, p)
    B.sph_forces(ctx, p)
    B.sph_hnet_set_weights(ctx, protocol_theta)
    dt = float(w.params["cfl"] * (p.h / p.vsig).min().item())
    for _ in range(2):
        B.sph_step(ctx, p, dt, use_hnet=B.SPH_HNET_SEED)
    snap = {f: getattr(p, f).clone() for f in ["x", "y", "z", "nnb", "id"] + B._FIELDS}
    s_plain = B.sph_step(ctx, p, dt)
    h_plain = p.in_original_order(["h"])["h"]
    for f, v in snap.items():
        getattr(p, f).copy_(v)
    s_learn = B.sph_step(ctx, p, dt, use_hnet=B.SPH_HNET_SEED)
    h_learn = p.in_original_order(["h"])["h"]
    ev_p, ev_l = s_plain["density"]["evaluations"], s_learn["density"]["evaluations"]
    print("evaluations plain", ev_p, "learned", ev_l, "ratio", ev_l / ev_p)
    assert np.max(np.abs(h_learn / h_plain - 1)) < 2 * w.params["h_tol"]
    assert ev_l < 0.8 * ev_p


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
    _check(op, g, t, 1e-5, 1e-4, exact_sets=False)
    nb = g["nnb"].mean()
    assert 90 < nb < 110                                 # ~100 neighbours with eta = 1.43971
