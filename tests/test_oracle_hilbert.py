"""Pins of the oracle's Hilbert keys (Sec. 2.1, Tree topology: the Hilbert
curve is the second space-filling curve beside Morton's).

The oracle follows the steps of Skilling's index construction.  These tests
check what makes the result a Hilbert curve and a valid octree key, without
re-running that construction: on small grids every index occurs once and
consecutive indices are face-neighbouring cells starting at the origin; at
the full 21 bits per axis the same adjacency holds around random cells (found
by probing the six face neighbours); the top 3k bits are the index of the
level-k cube on the order-k curve (so every octree cell is one contiguous key
range); keys of positions use the same cells as the Morton keys; and the
leaves defined on sorted Hilbert keys are the leaves defined on Morton keys.
"""
import itertools

import numpy as np
import pytest

TOP = (1 << 63) - 1


def _grid(bits):
    g = 1 << bits
    return np.array(list(itertools.product(range(g), repeat=3)), dtype=np.uint32).T


@pytest.mark.parametrize("bits", [1, 2, 3, 4, 5])
def test_small_grids_visit_every_cell_once_by_face_steps(orc, bits):
    c = _grid(bits)
    h = orc.hilbert_index(*c, bits=bits)
    assert np.array_equal(np.sort(h), np.arange(8 ** bits, dtype=np.uint64))
    walk = c[:, np.argsort(h)].astype(np.int64)
    steps = np.abs(np.diff(walk, axis=1))
    assert np.all(steps.sum(axis=0) == 1)            # one unit step along one axis
    assert np.all(walk[:, 0] == 0)                   # the curve starts at the origin cell


def test_full_resolution_face_adjacency(orc):
    rng = np.random.default_rng(11)
    n = 3000
    c = rng.integers(0, 1 << 21, size=(3, n)).astype(np.int64)
    c[:, 0] = 0                                      # the first cell
    c[:, 1] = [2 ** 21 - 1, 0, 0]                    # the last cell
    h = orc.hilbert_index(*c, bits=21).astype(np.uint64)
    nb = []
    for d in range(3):
        for s in (-1, 1):
            e = c.copy()
            e[d] += s
            inside = (e[d] >= 0) & (e[d] < 2 ** 21)
            e[d] = np.clip(e[d], 0, 2 ** 21 - 1)
            hn = orc.hilbert_index(*e, bits=21)
            nb.append(np.where(inside, hn, np.uint64(TOP + 1)))   # TOP + 1: no cell
    nb = np.stack(nb)
    nxt = (nb == h + np.uint64(1)).sum(axis=0)
    prv = (nb == h - np.uint64(1)).sum(axis=0)
    assert int(h[0]) == 0 and int(h[1]) == TOP
    assert np.all(nxt[h != np.uint64(TOP)] == 1)
    assert np.all(prv[h != np.uint64(0)] == 1)


def test_prefixes_are_the_coarse_curve(orc):
    rng = np.random.default_rng(12)
    c = rng.integers(0, 1 << 21, size=(3, 2000)).astype(np.uint32)
    h = orc.hilbert_index(*c, bits=21)
    for k in range(1, 21):
        coarse = orc.hilbert_index(*(c >> np.uint32(21 - k)), bits=k)
        assert np.array_equal(h >> np.uint64(3 * (21 - k)), coarse), k


def test_keys_use_the_morton_cells(orc):
    rng = np.random.default_rng(13)
    x, y, z = rng.random((3, 4000))
    lo, L = np.array([-0.3, 0.1, 0.2]), 1.9
    x, y, z = x * L + lo[0], y * L + lo[1], z * L + lo[2]
    x[:2] = [-9.0, 9.0]                              # outside: clamped to the boundary cells
    hk = orc.hilbert_keys(x, y, z, lo, L)
    mk = orc.morton_keys(x, y, z, lo, L)
    cells = [np.zeros(mk.size, dtype=np.uint64) for _ in range(3)]
    for b in range(21):                              # de-interleave the Morton key
        for d in range(3):
            cells[d] |= ((mk >> np.uint64(3 * b + d)) & np.uint64(1)) << np.uint64(b)
    ref = orc.hilbert_index(*cells, bits=21) | np.uint64(1 << 63)
    assert np.array_equal(hk, ref)
    assert np.all(hk >> np.uint64(63) == 1)


@pytest.mark.parametrize("leaf_size", [4, 32])
def test_leaves_do_not_depend_on_the_curve(orc, leaf_size):
    rng = np.random.default_rng(14)
    pts = np.concatenate([rng.random((3000, 3)), 0.61 + 0.002 * rng.random((300, 3))])
    ids = np.arange(len(pts), dtype=np.uint32)
    lv = {}
    for curve in ("morton", "hilbert"):
        k = orc.keys(pts[:, 0], pts[:, 1], pts[:, 2], np.zeros(3), 1.0, curve)
        perm = orc.sort_perm(k, ids)
        lv_sorted = orc.leaf_levels(k[perm], leaf_size)
        out = np.empty_like(lv_sorted)
        out[perm] = lv_sorted
        lv[curve] = out
    assert np.array_equal(lv["morton"], lv["hilbert"])
    assert lv["morton"].min() >= 1
