"""GPU parity of the density (Eqs. 7, 9) and force (Eqs. 5-6) passes against
the FP64 oracle: exact neighbour sets for the same positions and h, and the
floats to the tolerances of the workloads (1e-12 for the fixed-h lattice,
1e-10 for the variable-h Sedov blast in FP64)."""
import numpy as np
import pytest

import oracle
from gpu_helpers import need_gpu, to_oracle_params
from paper_2007_03097_gb300 import inputs

pytestmark = pytest.mark.gpu


def _sets(counts, offsets, idx, ids):
    """neighbour sets as sorted original ids, per particle (current order)"""
    return [np.sort(ids[idx[offsets[a]:offsets[a + 1]]]) for a in range(len(counts))]


def _run(w, fp64=True):
    B = need_gpu()
    ctx = B.Context(w.params, w.n)
    p = B.Particles.from_workload(w, fp64=fp64)
    B.sph_build_tree(ctx, p)
    ds = B.sph_density(ctx, p)
    fs = B.sph_forces(ctx, p)
    return B, ctx, p, ds, fs


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("wname,curve", [("lattice", "morton"), ("sedov", "morton"), ("polytrope", "morton"),
                                         ("sedov", "hilbert"), ("polytrope", "hilbert")])
def test_neighbour_sets_bit_exact(kind, wname, curve):
    w = {"lattice": lambda: inputs.lattice(16), "sedov": lambda: inputs.sedov(14),
         "polytrope": lambda: inputs.polytrope(6000, seed=4, precision="fp64")}[wname]()
    w.params["curve"] = curve
    B, ctx, p, _, _ = _run(w)
    g = p.numpy()
    op = to_oracle_params(oracle, w.params)
    counts, offsets, idx = B.sph_neighbors(ctx, p, kind)
    oc, oo, oi = oracle.neighbors(op, kind, g["x"], g["y"], g["z"], g["h"])
    assert np.array_equal(counts, oc)
    ids = np.arange(w.n)
    for a, (s1, s2) in enumerate(zip(_sets(counts, offsets, idx, ids), _sets(oc, oo, oi, ids))):
        assert np.array_equal(s1, s2), a


@pytest.mark.parametrize("wname,curve", [("lattice", "morton"), ("lattice", "hilbert"), ("polytrope", "morton"),
                                         ("polytrope", "hilbert")])
def test_neighbour_sets_of_large_sets(wname, curve):
    """The list walk starts at the nodes of grid cells a few levels below the
    root (the finest level whose cells cover a group's reach), looked up in a
    per-level cell table; cells inside a coarser leaf resolve to that leaf.
    A 64^3 periodic lattice (cells of level 2-3) and a 200,000-particle
    polytrope in its bounding cube (dense core: deep levels; sparse envelope:
    coarse leaves): the density and force sets of 4,000 sampled particles,
    including the extremes of each coordinate, equal the oracle's."""
    w = (inputs.lattice(64, jitter=0.3) if wname == "lattice"
         else inputs.polytrope(200000, seed=12, precision="fp64"))
    w.params["curve"] = curve
    B = need_gpu()
    ctx = B.Context(w.params, w.n)
    p = B.Particles.from_workload(w, fp64=True)
    B.sph_build_tree(ctx, p)
    B.sph_density(ctx, p)
    g = p.numpy()
    rng = np.random.default_rng(3)
    t = set(rng.choice(w.n, size=4000, replace=False).tolist())
    for c in ("x", "y", "z"):
        o = np.argsort(g[c])
        t.update(o[:20].tolist())
        t.update(o[-20:].tolist())
    t = np.array(sorted(t), dtype=np.int64)
    op = to_oracle_params(oracle, w.params)
    for kind in (0, 1):
        counts, offsets, idx = B.sph_neighbors(ctx, p, kind)
        oc, oo, oi = oracle.neighbors(op, kind, g["x"], g["y"], g["z"], g["h"], targets=t)
        assert np.array_equal(counts[t], oc)
        for k, a in enumerate(t):
            got = np.sort(idx[offsets[a]:offsets[a + 1]])
            assert np.array_equal(got, np.sort(oi[oo[k]:oo[k + 1]])), (kind, a)


def test_lattice_fixed_h_fp64():
    """16^3 jittered periodic lattice, M4, fixed h: floats to 1e-12."""
    w = inputs.lattice(16)
    B, ctx, p, ds, fs = _run(w)
    g = p.in_original_order()
    op = to_oracle_params(oracle, w.params)
    d = oracle.density(op, w.x, w.y, w.z, w.m, w.h)
    assert np.array_equal(g["nnb"], d.nnb)
    assert np.max(np.abs(g["rho"] / d.rho - 1)) < 1e-12
    assert np.max(np.abs(g["omega"] - d.drho_dh) / np.abs(d.drho_dh).max()) < 1e-12
    P, c = oracle.eos(op.gamma, d.rho, w.u)
    f = oracle.forces(op, w.x, w.y, w.z, w.vx, w.vy, w.vz, w.m, d.h, d.rho, P, c)
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(g[k] - getattr(f, k)) / f.S_a) < 1e-12, k
    assert np.max(np.abs(g["dudt"] - f.dudt)) < 1e-12 * max(1.0, np.abs(f.S_u).max())
    assert np.max(np.abs(g["vsig"] / f.vsig - 1)) < 1e-12
    assert np.max(np.abs(g["P"] / P - 1)) < 1e-12
    assert np.max(np.abs(g["P"] / ((op.gamma - 1) * g["rho"] * w.u) - 1)) < 1e-15      # EOS of the GPU's own rho
    assert fs["interactions"] == f.npairs
    assert ds["interactions"] == int(d.nnb.sum())


@pytest.mark.parametrize("curve", ["morton", "hilbert"])
def test_sedov_variable_h_fp64(curve):
    """Sedov blast (reduced to 16^3), Wendland C2, h-rho iteration to 1e-6;
    the particles in Morton or Hilbert order."""
    w = inputs.sedov(16)
    w.params["curve"] = curve
    rng = np.random.default_rng(1)
    w.vx, w.vy, w.vz = 0.1 * rng.standard_normal((3, w.n))     # exercise the viscosity
    B, ctx, p, ds, fs = _run(w)
    g = p.in_original_order()
    op = to_oracle_params(oracle, w.params)
    d = oracle.density(op, w.x, w.y, w.z, w.m, w.h)
    assert d.status == 0 and ds["status"] == 0
    assert np.max(np.abs(g["h"] / d.h - 1)) < 1e-10
    assert np.max(np.abs(g["rho"] / d.rho - 1)) < 1e-10
    P, c = oracle.eos(op.gamma, d.rho, w.u)
    f = oracle.forces(op, w.x, w.y, w.z, w.vx, w.vy, w.vz, w.m, d.h, d.rho, P, c)
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(g[k] - getattr(f, k)) / f.S_a) < 1e-10, k
    assert np.max(np.abs(g["dudt"] - f.dudt) / np.maximum(f.S_u, 1e-300)) < 1e-10
    assert np.max(np.abs(g["divv"] - f.divv)) < 1e-10 * np.abs(f.divv).max()
    assert np.max(np.abs(g["vsig"] / f.vsig - 1)) < 1e-10


@pytest.mark.parametrize("curve", ["morton", "hilbert"])
def test_mixed_precision_polytrope(curve):
    """n = 1 polytrope, FP32 pair arithmetic on two-float relative coordinates
    with FP64 positions: rho to 1e-5, a and du/dt to 1e-4 of their scale."""
    w = inputs.polytrope(20000, seed=11, precision="mixed")
    w.params["curve"] = curve
    rng = np.random.default_rng(2)
    w.vx, w.vy, w.vz = 0.05 * rng.standard_normal((3, w.n))
    B, ctx, p, ds, fs = _run(w, fp64=False)
    g = p.in_original_order()
    op = to_oracle_params(oracle, w.params)
    d = oracle.density(op, w.x, w.y, w.z, w.m, w.h)
    assert np.max(np.abs(g["rho"] / d.rho - 1)) < 1e-5
    assert np.max(np.abs(g["h"] / d.h - 1)) < 1e-5
    P, c = oracle.eos(op.gamma, d.rho, w.u)
    f = oracle.forces(op, w.x, w.y, w.z, w.vx, w.vy, w.vz, w.m, d.h, d.rho, P, c)
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(g[k] - getattr(f, k)) / f.S_a) < 1e-4, k
    assert np.max(np.abs(g["dudt"] - f.dudt) / np.maximum(f.S_u, 1e-30)) < 1e-4


@pytest.mark.parametrize("precision,tol_rho,tol_a", [("mixed", 1e-5, 1e-4), ("fp64", 1e-10, 1e-10)])
def test_large_source_unions(precision, tol_rho, tol_a):
    """Many neighbours (eta = 2.2, ~470 per particle): each group's source
    union holds well over the 448 sources a warp stages at once, so the mixed
    sweep runs in several chunks; both precisions against the oracle."""
    w = inputs.lattice(14, jitter=0.2, kernel=1, h_factor=2.2, fixed_h=False, precision=precision)
    w.params["nb_capacity"] = 1024 * w.n                 # ~440 list slots per particle, beyond the default
    rng = np.random.default_rng(8)
    w.vx, w.vy, w.vz = 0.2 * rng.standard_normal((3, w.n))
    B, ctx, p, ds, fs = _run(w, fp64=precision == "fp64")
    info = B.sph_list_info(ctx)
    _, ng = B.sph_tree_info(ctx)
    assert info["union_used"] / ng > 448
    g = p.in_original_order()
    op = to_oracle_params(oracle, w.params)
    d = oracle.density(op, w.x, w.y, w.z, w.m, w.h)
    assert np.max(np.abs(g["rho"] / d.rho - 1)) < tol_rho
    assert np.max(np.abs(g["h"] / d.h - 1)) < tol_rho
    P, c = oracle.eos(op.gamma, d.rho, w.u)
    f = oracle.forces(op, w.x, w.y, w.z, w.vx, w.vy, w.vz, w.m, d.h, d.rho, P, c)
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(g[k] - getattr(f, k)) / f.S_a) < tol_a, k
