"""GPU parity of the tree stage (Sec. 2.1, Tree topology): Morton and Hilbert
keys and the (key, id) sort permutation bit-exact against the oracle, the
in-place permutation of the particle arrays, and the octree leaves against the
leaf definition evaluated by the oracle, on either curve."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import need_gpu, to_oracle_params
from paper_2007_03097_gb300 import inputs

pytestmark = pytest.mark.gpu


def _cloud(n, seed, periodic):
    rng = np.random.default_rng(seed)
    if periodic:
        w = inputs.lattice(4, jitter=0.0)
        w = w.subset(np.zeros(n, dtype=np.int64))
        w.x, w.y, w.z = rng.random((3, n))
    else:
        w = inputs.polytrope(n, seed=seed, precision="fp64")
    return w


@pytest.mark.parametrize("curve", ["morton", "hilbert"])
@pytest.mark.parametrize("n,periodic", [(1, True), (37, True), (4097, True), (50000, False), (70001, True)])
def test_keys_bit_exact(n, periodic, curve):
    B = need_gpu()
    w = _cloud(n, 1, periodic)
    w.params["curve"] = curve
    if n > 2:                                            # the corner cells of the key grid
        w.x[:2], w.y[:2], w.z[:2] = (0.0, 1.0 - 1e-12), (0.0, 1.0 - 1e-12), (0.0, 1.0 - 1e-12)
    ctx = B.Context(w.params, n)
    p = B.Particles.from_workload(w, fp64=True)
    keys, dom = B.sph_morton_keys(ctx, p)
    op = to_oracle_params(oracle, w.params)
    lo, L = oracle.domain(w.x, w.y, w.z, op)
    assert np.array_equal(dom, np.array([*lo, L]))
    ref = oracle.keys(w.x, w.y, w.z, lo, L, curve)
    assert np.array_equal(keys, ref)


@pytest.mark.parametrize("n", [1, 2, 4095, 4096, 4097, 100003])
def test_sort_permutation_bit_exact(n):
    B = need_gpu()
    rng = np.random.default_rng(n)
    pool = (rng.integers(0, 1 << 62, size=n // 4 + 1, dtype=np.int64).astype(np.uint64)) | np.uint64(1 << 63)
    keys = pool[rng.integers(0, pool.size, size=n)]      # short runs of equal keys
    ids = rng.permutation(n).astype(np.uint32)
    ctx = B.Context({}, n)
    kt = torch.from_numpy(keys.view(np.int64)).cuda()
    it = torch.from_numpy(ids.view(np.int32)).cuda()
    perm = B.sph_sort_keys(ctx, kt, it).cpu().numpy().view(np.uint32)
    assert np.array_equal(perm, oracle.sort_perm(keys, ids))


def test_sort_rejects_long_equal_key_runs():
    B = need_gpu()
    n = 1000
    keys = np.full(n, (1 << 63) | 12345, dtype=np.uint64)
    ctx = B.Context({}, n)
    with pytest.raises(B.SphError) as e:
        B.sph_sort_keys(ctx, torch.from_numpy(keys.view(np.int64)).cuda(), None)
    assert e.value.code == B.SPH_ERR_CAPACITY


def test_sort_permutation_many_duplicates():
    B = need_gpu()
    rng = np.random.default_rng(5)
    n = 20000
    keys = (rng.integers(0, 1500, size=n).astype(np.uint64)) | np.uint64(1 << 63)
    ids = rng.permutation(n).astype(np.uint32)
    ctx = B.Context({}, n)
    perm = B.sph_sort_keys(ctx, torch.from_numpy(keys.view(np.int64)).cuda(),
                           torch.from_numpy(ids.view(np.int32)).cuda()).cpu().numpy().view(np.uint32)
    assert np.array_equal(perm, oracle.sort_perm(keys, ids))


@pytest.mark.parametrize("name,leaf_size,curve", [("lattice", 32, "morton"), ("polytrope", 32, "morton"),
                                                  ("polytrope", 8, "morton"), ("lattice", 32, "hilbert"),
                                                  ("polytrope", 32, "hilbert"), ("polytrope", 8, "hilbert")])
def test_build_tree_order_and_leaves(name, leaf_size, curve):
    B = need_gpu()
    w = inputs.lattice(20, jitter=0.1) if name == "lattice" else inputs.polytrope(30000, seed=9, precision="fp64")
    w.params["leaf_size"] = leaf_size
    w.params["curve"] = curve
    rng = np.random.default_rng(0)
    w.u = rng.random(w.n) + 0.5                          # a field to follow through the permutation
    ctx = B.Context(w.params, w.n)
    p = B.Particles.from_workload(w, fp64=True)
    ids = rng.permutation(w.n).astype(np.uint32)
    p.id.copy_(torch.from_numpy(ids.view(np.int32)))
    B.sph_build_tree(ctx, p)
    op = to_oracle_params(oracle, w.params)
    lo, L = oracle.domain(w.x, w.y, w.z, op)
    keys = oracle.keys(w.x, w.y, w.z, lo, L, curve)
    perm = oracle.sort_perm(keys, ids)
    g = p.numpy()
    assert np.array_equal(g["id"], ids[perm])
    assert np.array_equal(g["x"], w.x[perm]) and np.array_equal(g["u"], w.u[perm])
    lvl = oracle.leaf_levels(keys[perm], leaf_size)
    lb, lv = B.sph_export_leaves(ctx)
    # leaf starts by definition: level changes or prefix at that level changes
    sk = keys[perm]
    start = [0]
    for i in range(1, w.n):
        L_i = int(lvl[i])
        if (int(sk[i]) >> (63 - 3 * L_i)) != (int(sk[i - 1]) >> (63 - 3 * L_i)):
            start.append(i)
    assert np.array_equal(lb[:-1], np.array(start)) and lb[-1] == w.n
    assert np.array_equal(lv, lvl[np.array(start)])
    nl, ng = B.sph_tree_info(ctx)
    assert nl == len(start) and 1 <= ng <= w.n


@pytest.mark.parametrize("moved,curve", [(0, "morton"), (1, "morton"), (50, "morton"), (3000, "morton"),
                                         (20000, "morton"), (50, "hilbert"), (3000, "hilbert")])
def test_rebuild_of_nearly_sorted_particles(moved, curve):
    """A rebuild after small moves (the state of every step after the first)
    finds most particles in place and moves only the misplaced ones; the
    order must still be the (key, id) sort of the current keys.  Large moves
    take the full sort."""
    B = need_gpu()
    w = inputs.lattice(24, jitter=0.1)                  # 13,824 particles
    rng = np.random.default_rng(moved + 11)
    w.u = rng.random(w.n) + 0.5
    w.params["curve"] = curve
    ctx = B.Context(w.params, w.n)
    p = B.Particles.from_workload(w, fp64=True)
    B.sph_build_tree(ctx, p)                             # key order of the initial state
    g = p.numpy()
    x, y, z = g["x"].copy(), g["y"].copy(), g["z"].copy()
    k = min(moved, w.n)
    sel = rng.choice(w.n, size=k, replace=False)
    spacing = 1.0 / 24
    x[sel] = np.mod(x[sel] + rng.uniform(-1.5, 1.5, k) * spacing, 1.0)
    y[sel] = np.mod(y[sel] + rng.uniform(-1.5, 1.5, k) * spacing, 1.0)
    if k > 1:                                            # two particles on one key: ties by id
        x[sel[1]], y[sel[1]], z[sel[1]] = x[sel[0]], y[sel[0]], z[sel[0]]
    for f, v in (("x", x), ("y", y), ("z", z)):
        getattr(p, f).copy_(torch.from_numpy(v))
    B.sph_build_tree(ctx, p)
    op = to_oracle_params(oracle, w.params)
    lo, L = oracle.domain(x, y, z, op)
    keys = oracle.keys(x, y, z, lo, L, curve)
    perm = oracle.sort_perm(keys, g["id"])
    h = p.numpy()
    assert np.array_equal(h["id"], g["id"][perm])
    assert np.array_equal(h["x"], x[perm]) and np.array_equal(h["y"], y[perm])
    assert np.array_equal(h["u"], g["u"][perm])
    lb, _ = B.sph_export_leaves(ctx)
    assert lb[-1] == w.n and np.all(np.diff(lb) > 0)


def test_fig1_quadtree_leaves():
    """The ten particles of Fig. 1 (Sec. 2.1, tests/golden/fig1_quadtree.txt)
    in the unit box at z = 0 with leaf_size 1: the library's order is the
    figure's Z-order and its leaves are the figure's cells (level = digits
    below the leading 1)."""
    from helpers import fig1_quadtree
    B = need_gpu()
    labels, x, y, _, path = fig1_quadtree()
    w = _cloud(len(labels), 0, True)
    w.x, w.y, w.z = x, y, np.zeros_like(x)
    w.params["leaf_size"] = 1
    ctx = B.Context(w.params, w.n)
    p = B.Particles.from_workload(w, fp64=True)
    B.sph_build_tree(ctx, p)
    g = p.numpy()
    got = [labels[i] for i in g["id"]]
    assert got == sorted(labels, key=lambda c: (path.index(c[:3]) if c[:3] in path else path.index(c[:2]), c))
    lb, lv = B.sph_export_leaves(ctx)
    assert np.array_equal(lb, np.arange(len(labels) + 1))
    assert list(lv) == [len(c) - 1 for c in got]


@pytest.mark.parametrize("cluster,curve", [(0, "morton"), (0, "hilbert"), (40, "morton"), (300, "morton"),
                                           (300, "hilbert")])
def test_build_tree_order_with_shared_top_key_bits(cluster, curve):
    """The build sorts on the top 32 key bits and then orders each run of
    equal top halves by (key, id); a run longer than 64 sends it to a sort on
    all bits.  Uniform particles plus pairs and triples closer than 2^-12 of
    the box (short runs, one pair on the same key: id order), and a cluster of
    `cluster` particles inside one cell of side 2^-12 (a run of that length):
    the order must be the (key, id) sort of the oracle's keys, with the
    leaves of the leaf definition."""
    B = need_gpu()
    rng = np.random.default_rng(cluster + (7 if curve == "hilbert" else 0))
    n0 = 20000
    x, y, z = rng.random((3, n0))
    eps = 2.0 ** -14
    for k in range(0, 300, 3):                           # pairs and triples around particle k
        for j in (1, 2):
            if j == 2 and k % 2:
                continue
            x[k + j], y[k + j], z[k + j] = x[k] + j * eps, y[k], z[k] + eps * rng.random()
    x[400], y[400], z[400] = x[399], y[399], z[399]     # two particles on one key
    if cluster:
        c = (np.floor(rng.random(3) * 0.9 * 2 ** 11) + 0.25) / 2 ** 11      # inside one level-11 cell
        cx, cy, cz = (c + rng.random((3, cluster)).T * 2.0 ** -12).T
        x, y, z = np.concatenate([x, cx]), np.concatenate([y, cy]), np.concatenate([z, cz])
    n = x.size
    w = _cloud(n, 0, True)
    w.x, w.y, w.z = np.mod(x, 1.0), np.mod(y, 1.0), np.mod(z, 1.0)
    w.params["curve"] = curve
    w.params["leaf_size"] = 8
    w.u = rng.random(n) + 0.5
    ctx = B.Context(w.params, n)
    p = B.Particles.from_workload(w, fp64=True)
    ids = rng.permutation(n).astype(np.uint32)
    p.id.copy_(torch.from_numpy(ids.view(np.int32)))
    B.sph_build_tree(ctx, p)
    op = to_oracle_params(oracle, w.params)
    lo, L = oracle.domain(w.x, w.y, w.z, op)
    keys = oracle.keys(w.x, w.y, w.z, lo, L, curve)
    top = keys >> np.uint64(32)
    runs = np.diff(np.flatnonzero(np.diff(np.concatenate([[-1], np.sort(top).astype(np.float64), [-1]])) != 0))
    assert runs.max() >= (cluster if cluster else 2)     # the case is the one named
    perm = oracle.sort_perm(keys, ids)
    g = p.numpy()
    assert np.array_equal(g["id"], ids[perm])
    assert np.array_equal(g["x"], w.x[perm]) and np.array_equal(g["u"], w.u[perm])
    lvl = oracle.leaf_levels(keys[perm], 8)
    sk = keys[perm]
    start = [0] + [i for i in range(1, n)
                   if (int(sk[i]) >> (63 - 3 * int(lvl[i]))) != (int(sk[i - 1]) >> (63 - 3 * int(lvl[i])))]
    lb, lv = B.sph_export_leaves(ctx)
    assert np.array_equal(lb[:-1], np.array(start)) and lb[-1] == n
    assert np.array_equal(lv, lvl[np.array(start)])
