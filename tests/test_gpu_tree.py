"""GPU parity of the tree stage (Sec. 2.1, Tree topology): Morton keys and the
(key, id) sort permutation bit-exact against the oracle, the in-place
permutation of the particle arrays, and the octree leaves against the leaf
definition evaluated by the oracle."""
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


@pytest.mark.parametrize("n,periodic", [(1, True), (37, True), (4097, True), (50000, False), (70001, True)])
def test_morton_keys_bit_exact(n, periodic):
    B = need_gpu()
    w = _cloud(n, 1, periodic)
    ctx = B.Context(w.params, n)
    p = B.Particles.from_workload(w, fp64=True)
    keys, dom = B.sph_morton_keys(ctx, p)
    op = to_oracle_params(oracle, w.params)
    lo, L = oracle.domain(w.x, w.y, w.z, op)
    assert np.array_equal(dom, np.array([*lo, L]))
    ref = oracle.morton_keys(w.x, w.y, w.z, lo, L)
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


@pytest.mark.parametrize("name,leaf_size", [("lattice", 32), ("polytrope", 32), ("polytrope", 8)])
def test_build_tree_order_and_leaves(name, leaf_size):
    B = need_gpu()
    w = inputs.lattice(20, jitter=0.1) if name == "lattice" else inputs.polytrope(30000, seed=9, precision="fp64")
    w.params["leaf_size"] = leaf_size
    rng = np.random.default_rng(0)
    w.u = rng.random(w.n) + 0.5                          # a field to follow through the permutation
    ctx = B.Context(w.params, w.n)
    p = B.Particles.from_workload(w, fp64=True)
    ids = rng.permutation(w.n).astype(np.uint32)
    p.id.copy_(torch.from_numpy(ids.view(np.int32)))
    B.sph_build_tree(ctx, p)
    op = to_oracle_params(oracle, w.params)
    lo, L = oracle.domain(w.x, w.y, w.z, op)
    keys = oracle.morton_keys(w.x, w.y, w.z, lo, L)
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
