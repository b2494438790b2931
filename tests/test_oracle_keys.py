"""Pins of the oracle's Morton keys, sort permutation and leaf levels
(Sec. 2.1, Tree topology and Fig. 1).

The key encoder in the oracle is a bit loop; these tests check it against
hand-known keys, an independent decoder, the classic "most significant
differing bit" Z-order comparison (which never interleaves bits), numpy's
lexsort, and the leaf definition checked by brute force on small sets.
"""
import functools

import numpy as np
import pytest


def _cells(keys):
    """Independent decoder: de-interleave the low 63 bits into (ix, iy, iz)."""
    k = np.asarray(keys, dtype=np.uint64)
    out = [np.zeros(k.size, dtype=np.uint64) for _ in range(3)]
    for b in range(21):
        for d in range(3):
            out[d] |= ((k >> np.uint64(3 * b + d)) & np.uint64(1)) << np.uint64(b)
    return out


def _point(ix, iy, iz):
    """Centre of cell (ix, iy, iz) in the unit domain."""
    s = 2.0 ** -21
    return (np.array([ix]) + 0.5) * s, (np.array([iy]) + 0.5) * s, (np.array([iz]) + 0.5) * s


def test_known_keys(orc):
    lo = np.zeros(3)
    cases = {(0, 0, 0): 1 << 63, (1, 0, 0): (1 << 63) | 1, (0, 1, 0): (1 << 63) | 2,
             (0, 0, 1): (1 << 63) | 4, (2, 0, 0): (1 << 63) | 8, (1, 1, 1): (1 << 63) | 7,
             (2 ** 21 - 1,) * 3: (1 << 64) - 1}
    for cell, key in cases.items():
        assert int(orc.morton_keys(*_point(*cell), lo, 1.0)[0]) == key


def test_decode_roundtrip_and_clamp(orc):
    rng = np.random.default_rng(0)
    x, y, z = rng.random((3, 5000))
    lo = np.array([-0.1, 0.2, 0.0])
    L = 1.7
    keys = orc.morton_keys(x * L + lo[0], y * L + lo[1], z * L + lo[2], lo, L)
    assert np.all(keys >> np.uint64(63) == 1)
    for d, (c, u) in enumerate(zip(_cells(keys), (x, y, z))):
        # the decoded cell holds the point (up to rounding at a cell face)
        assert np.all(np.abs(c.astype(np.float64) - np.floor(u * 2 ** 21)) <= 1)
    # out-of-domain coordinates clamp to the boundary cells
    k = orc.morton_keys(np.array([-5.0, 5.0]), np.array([0.5, 0.5]), np.array([0.5, 0.5]), np.zeros(3), 1.0)
    cx = _cells(k)[0]
    assert int(cx[0]) == 0 and int(cx[1]) == 2 ** 21 - 1


def _z_less(a, b):
    """Z-order comparison without interleaving: the axis whose coordinates
    differ in the most significant bit decides (ties in that bit position go
    to the higher axis, z > y > x, matching x in the lowest bit)."""
    best_axis, best_msb = -1, -1
    for d in range(3):
        x = int(a[d]) ^ int(b[d])
        if x == 0:
            continue
        msb = x.bit_length() - 1
        if msb >= best_msb:
            best_axis, best_msb = d, msb
    if best_axis < 0:
        return 0
    return -1 if a[best_axis] < b[best_axis] else 1


def test_key_order_is_z_order(orc):
    rng = np.random.default_rng(1)
    cells = rng.integers(0, 2 ** 21, size=(400, 3))
    cells[:50] = rng.integers(0, 8, size=(50, 3))             # many shared high bits
    s = 2.0 ** -21
    keys = orc.morton_keys((cells[:, 0] + 0.5) * s, (cells[:, 1] + 0.5) * s, (cells[:, 2] + 0.5) * s,
                           np.zeros(3), 1.0)
    order_keys = np.argsort(keys, kind="stable")
    order_z = sorted(range(len(cells)), key=functools.cmp_to_key(lambda i, j: _z_less(cells[i], cells[j]) or (i - j)))
    assert list(order_keys) == order_z


def test_sort_perm_matches_lexsort(orc):
    rng = np.random.default_rng(2)
    keys = rng.integers(0, 50, size=3000).astype(np.uint64) | np.uint64(1 << 63)   # many equal keys
    ids = rng.permutation(3000).astype(np.uint32)
    perm = orc.sort_perm(keys, ids)
    ref = np.lexsort((ids, keys))
    assert np.array_equal(perm, ref.astype(np.uint32))


def _leaf_brute(keys, leaf_size):
    """Brute force: for each particle test every level by counting all keys."""
    n = len(keys)
    out = []
    for i in range(n):
        lvl_found = -1
        for lvl in range(22):
            sh = 63 - 3 * lvl
            p = int(keys[i]) >> sh
            cnt = sum(1 for j in range(n) if (int(keys[j]) >> sh) == p)
            if cnt <= leaf_size:
                lvl_found = lvl
                break
        out.append(lvl_found)
    return np.array(out)


@pytest.mark.parametrize("leaf_size", [4, 32])
def test_leaf_levels_by_brute_force(orc, leaf_size):
    rng = np.random.default_rng(3)
    pts = np.concatenate([rng.random((150, 3)), 0.3 + 0.01 * rng.random((60, 3))])   # a dense clump
    keys = np.sort(orc.morton_keys(pts[:, 0], pts[:, 1], pts[:, 2], np.zeros(3), 1.0))
    lv = orc.leaf_levels(keys, leaf_size)
    assert np.array_equal(lv, _leaf_brute(keys, leaf_size))
    # leaves partition the particles into contiguous runs of at most leaf_size
    start = np.ones(keys.size, dtype=bool)
    for i in range(1, keys.size):
        L = int(lv[i])
        start[i] = (int(keys[i]) >> (63 - 3 * L)) != (int(keys[i - 1]) >> (63 - 3 * L))
    b = np.nonzero(start)[0]
    sizes = np.diff(np.append(b, keys.size))
    assert sizes.max() <= leaf_size


def test_fig1_quadtree(orc):
    """Sec. 2.1, Fig. 1 (tests/golden/fig1_quadtree.txt): with z = 0 every
    3-bit level of a key is the figure's base-4 digit, so the leading 1 and
    the octal digits below it spell the label of each particle's cell; the
    particles sort in the figure's Z-order path; and refining until every
    particle is alone in its cell (leaf_size 1) gives the figure's leaves and
    subdivided cells."""
    from helpers import fig1_quadtree
    labels, x, y, refined, path = fig1_quadtree()
    keys = orc.morton_keys(x, y, np.zeros_like(x), np.zeros(3), 1.0)
    for lab, k in zip(labels, keys):
        assert "1" + "".join(str((int(k) >> (63 - 3 * l)) & 7) for l in range(1, len(lab))) == lab
    order = np.argsort(keys)
    rank = {c: i for i, c in enumerate(path)}
    seq = [rank[lab[:3]] if lab[:3] in rank else rank[lab[:2]] for lab in np.array(labels)[order]]
    assert seq == sorted(seq)
    sk = keys[order]
    lv = orc.leaf_levels(sk, 1)
    assert [len(lab) - 1 for lab in np.array(labels)[order]] == list(lv)
    def label(k, level):
        return "1" + "".join(str((int(k) >> (63 - 3 * l)) & 7) for l in range(1, level + 1))
    inner = {label(k, a) for k, leaf in zip(sk, lv) for a in range(int(leaf))}
    assert inner == set(refined)
