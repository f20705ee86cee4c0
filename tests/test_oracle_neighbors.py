"""Pins of the oracle's neighbour search (CPU only).

The paper needs, for the particle-particle contact constraint, the pairs of
particles of *different object groups* that may touch (Sec. III-A, constraint
(2); the particle contact step of Algorithm 1) but does not say how they are found.  The oracle's
definition is the O(N^2) FP32 predicate; its hashed-grid search must return
exactly the same sets, and both are checked against an independent library
range query (scipy's k-d tree in FP64) away from the rounding band at R_n.
"""
import numpy as np
import pytest

from paper_2603_14634_gb300 import scenes


def _random_bodies(rng, n_bodies, per_body, box=0.6):
    pos = rng.random((n_bodies * per_body, 3)).astype(np.float32) * box
    body = np.repeat(np.arange(n_bodies, dtype=np.int32), per_body)
    return pos, body


def _csr_sets(off, idx):
    return [tuple(idx[off[p]:off[p + 1]]) for p in range(len(off) - 1)]


def test_constants_follow_definition(orc):
    Rn, Rn2, h, inv_h = orc.nbr_constants(0.05)
    assert Rn == np.float32(2.2 * 0.05)
    assert Rn2 == np.float32(Rn) * np.float32(Rn)
    assert h == np.float32(np.float64(Rn) * (1 + 2.0 ** -10))
    assert inv_h == np.float32(1.0 / np.float64(h))
    assert h > Rn


def test_table_size_power_of_two(orc):
    for n, t in [(1, 2), (2, 4), (3, 8), (64, 128), (65, 256), (8000, 16384)]:
        assert orc.table_size(n) == t


def test_cell_hash_matches_teschner_definition(orc):
    """bucket = (ix*73856093 ^ iy*19349663 ^ iz*83492791) mod 2^32 & (T-1)
    (Teschner et al. 2003), cell = floor(x * inv_h) in FP32."""
    _, _, _, inv_h = orc.nbr_constants(0.05)
    rng = np.random.default_rng(3)
    x = ((rng.random((50, 3)) - 0.5) * 20).astype(np.float32)
    keys = orc.cell_keys(x, 0.05)
    T = orc.table_size(50)
    for p in range(50):
        c = [int(np.floor(np.float32(x[p, k]) * np.float32(inv_h))) for k in range(3)]
        h = ((c[0] * 73856093) ^ (c[1] * 19349663) ^ (c[2] * 83492791)) & 0xFFFFFFFF
        assert keys[p] == (h & (T - 1))


def test_sorted_keys_stable(orc):
    rng = np.random.default_rng(0)
    x = (rng.random((3000, 3)) * 2).astype(np.float32)
    sk, si = orc.sorted_keys(x, 0.05)
    keys = orc.cell_keys(x, 0.05)
    order = np.lexsort((np.arange(len(keys)), keys))     # library stable sort
    np.testing.assert_array_equal(si, order.astype(np.uint32))
    np.testing.assert_array_equal(sk, keys[order])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_grid_equals_brute_force_random(orc, seed):
    rng = np.random.default_rng(seed)
    pos, body = _random_bodies(rng, 40, 50)
    a = orc.neighbors(pos, body, 0.05, "grid")
    b = orc.neighbors(pos, body, 0.05, "brute")
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert a[1].size > 0


def test_grid_equals_brute_force_lattice_scene(orc):
    sc = scenes.random_bodies_scene(seed=1, num_bodies=12)
    # squeeze the bodies together so that many cross-body pairs exist
    pos = (sc.pos * np.float32(0.55)).astype(np.float32)
    body = orc.body_index(sc.body_off)
    a = orc.neighbors(pos, body, sc.radius, "grid")
    b = orc.neighbors(pos, body, sc.radius, "brute")
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert a[1].size > 100


def test_boundary_pairs_exact(orc):
    """Pairs placed exactly at, just inside and just outside R_n, and
    particles on cell faces, decided by the FP32 predicate d2 < Rn^2."""
    Rn, Rn2, h, inv_h = orc.nbr_constants(0.05)
    pts, bodies = [], []
    k = 0
    for base in (0.0, float(h), 3 * float(h), -2 * float(h)):
        for gap in (np.nextafter(Rn, np.float32(0)), Rn, np.nextafter(Rn, np.float32(1))):
            p = np.array([base, 0.37, 0.11], dtype=np.float32)
            q = p.copy()
            q[0] = np.float32(p[0] + gap)
            pts += [p, q]
            bodies += [k, k + 1]
            k += 2
    pos = np.stack(pts).astype(np.float32)
    # move groups far apart so only the intended pairs interact
    pos[:, 1] += np.repeat(np.arange(len(pts) // 2, dtype=np.float32), 2) * 1.0
    body = np.array(bodies, dtype=np.int32)
    a = orc.neighbors(pos, body, 0.05, "grid")
    b = orc.neighbors(pos, body, 0.05, "brute")
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[0], b[0])
    # expected decision from the FP32 predicate evaluated here with numpy
    for i in range(0, len(pts), 2):
        d = pos[i + 1] - pos[i]
        d2 = np.float32(np.float32(d[0] * d[0]) + np.float32(d[1] * d[1])) + np.float32(d[2] * d[2])
        has = (i + 1) in a[1][a[0][i]:a[0][i + 1]]
        assert has == bool(np.float32(d2) < np.float32(Rn2))


def test_same_body_never_listed_and_symmetric(orc):
    rng = np.random.default_rng(5)
    pos, body = _random_bodies(rng, 10, 60, box=0.4)
    off, idx = orc.neighbors(pos, body, 0.05)
    sets = _csr_sets(off, idx)
    for p, s in enumerate(sets):
        assert list(s) == sorted(s)
        for q in s:
            assert body[q] != body[p]
            assert p in sets[q]


def test_against_kdtree_range_query(orc):
    """Independent check with scipy's k-d tree (FP64): every pair clearly
    inside R_n is listed and none clearly outside."""
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(11)
    pos, body = _random_bodies(rng, 30, 80, box=0.8)
    Rn = orc.nbr_constants(0.05)[0]
    off, idx = orc.neighbors(pos, body, 0.05)
    sets = [set(s) for s in _csr_sets(off, idx)]
    tree = spatial.cKDTree(pos.astype(np.float64))
    inner = tree.query_pairs(Rn * (1 - 1e-5), output_type="ndarray")
    outer = tree.query_pairs(Rn * (1 + 1e-5), output_type="ndarray")
    for p, q in inner:
        if body[p] != body[q]:
            assert q in sets[p] and p in sets[q]
    outer_set = {(min(p, q), max(p, q)) for p, q in outer}
    for p, s in enumerate(sets):
        for q in s:
            assert (min(p, q), max(p, q)) in outer_set


def test_empty_and_single(orc):
    off, idx = orc.neighbors(np.zeros((0, 3), np.float32), np.zeros(0, np.int32), 0.05)
    assert off.tolist() == [0] and idx.size == 0
    off, idx = orc.neighbors(np.zeros((1, 3), np.float32), np.zeros(1, np.int32), 0.05)
    assert off.tolist() == [0, 0] and idx.size == 0
