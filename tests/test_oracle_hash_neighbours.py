"""Pins of the oracle's bucket hash, stable sort, bucket ranges and neighbour search (Sec. I).

The method *is* these definitions: bucket side 2h, hash = x-fastest linear bucket index, particles
outside the fixed grid get the garbage hash (the bucket count), a stable sort by hash, and a
neighbour search restricted to the particle's bucket and the 26 around it.
"""
import itertools

import numpy as np
import pytest

from oracle import orc
from paper_2310_03596_gb300 import scenes


def _params(lo=(0.0, 0.0, 0.0), dims=(4, 3, 2), h=0.5, walls=()):
    s = scenes.cube_impact(n_side=2)
    s.grid_lo, s.grid_dims, s.h, s.walls = lo, dims, h, list(walls)
    return orc.params_of(s)


def test_hash_closed_form():
    # bucket side 2h = 1: coordinates are the integer parts; x fastest
    P = _params()
    pts = np.array([[0.0, 0.0, 0.0], [0.999, 0.0, 0.0], [1.0, 0.0, 0.0], [3.5, 2.5, 1.5],
                    [2.2, 1.7, 0.1], [4.0, 0.0, 0.0], [-1e-12, 0.0, 0.0], [0.0, 3.0, 0.0],
                    [0.5, 0.5, 2.0], [np.nan, 0.0, 0.0]])
    want = [0, 0, 1, 3 + 4 * (2 + 3 * 1), 2 + 4 * 1, 24, 24, 24, 24, 24]
    got = orc.hash_keys(P, pts[:, 0], pts[:, 1], pts[:, 2])
    assert got.tolist() == want


def test_sort_is_stable_argsort():
    rng = np.random.default_rng(5)
    key = rng.integers(0, 50, size=5000).astype(np.uint32)
    perm = orc.sort_order(key)
    assert np.array_equal(perm, np.argsort(key, kind="stable"))


def test_cell_ranges_match_searchsorted():
    rng = np.random.default_rng(6)
    key = np.sort(rng.integers(0, 200, size=3000)).astype(np.uint32)
    key[-7:] = 200  # garbage tail
    st, en = orc.cell_ranges(key, 200)
    for c in range(200):
        a, b = np.searchsorted(key, c, "left"), np.searchsorted(key, c, "right")
        if a == b:
            assert st[c] == 0 and en[c] == 0
        else:
            assert (st[c], en[c]) == (a, b)


def _sorted_rows(lst, cnt):
    return [sorted(lst[i, : cnt[i]].tolist()) for i in range(len(cnt))]


@pytest.mark.parametrize("walls", [[], [(2, 0.0)], [(0, 0.0), (2, 0.0)]])
def test_bucket_search_equals_brute_force(walls):
    s = scenes.cube_impact(n_side=12)
    s.walls = walls
    P = orc.params_of(s)
    x, y, z = s.pos.T
    c1, l1 = orc.neighbours(P, x, y, z)
    c2, l2 = orc.neighbours(P, x, y, z, brute=True)
    assert np.array_equal(c1, c2)
    assert _sorted_rows(l1, c1) == _sorted_rows(l2, c2)


def test_bucket_search_equals_brute_force_random_cloud():
    # irregular density (clumps and voids) and particles outside the grid
    rng = np.random.default_rng(11)
    h = 0.1
    pts = np.concatenate([rng.random((1500, 3)), 0.5 + 0.05 * rng.standard_normal((500, 3)),
                          rng.random((20, 3)) * 3.0 - 1.0])
    s = scenes.cube_impact(n_side=2)
    s.grid_lo, s.grid_dims, s.h, s.walls = (0.0, 0.0, 0.0), (5, 5, 5), h, [(1, 0.0)]
    P = orc.params_of(s)
    c1, l1 = orc.neighbours(P, *pts.T, cap=1024)
    c2, l2 = orc.neighbours(P, *pts.T, cap=1024, brute=True)
    assert np.array_equal(c1, c2)
    assert _sorted_rows(l1, c1) == _sorted_rows(l2, c2)
    # outside-grid particles interact with nobody
    key = orc.hash_keys(P, *pts.T)
    assert (c1[key == 125] == 0).all()


def test_interior_count_is_80_on_jittered_lattice():
    # lattice points k != 0 with |k|^2 < (2h/dx)^2 = 2.6^2 = 6.76; the jitter (1% dx) cannot cross
    # from |k|^2 = 6 to 6.76 or from 7 down to 6.76
    want = sum(1 for k in itertools.product(range(-3, 4), repeat=3)
               if k != (0, 0, 0) and k[0] ** 2 + k[1] ** 2 + k[2] ** 2 < 6.76)
    assert want == 80
    s = scenes.cube_impact(n_side=16)
    s.walls = []
    P = orc.params_of(s)
    cnt, _ = orc.neighbours(P, *s.pos.T)
    idx = np.rint(s.pos / s.dx - 0.5).astype(int)
    interior = ((idx >= 3) & (idx <= 12)).all(axis=1)
    assert interior.sum() == 1000
    assert (cnt[interior] == 80).all()
    assert cnt.max() == 80


def test_wall_images_present_only_near_wall():
    s = scenes.cube_impact(n_side=8)
    P = orc.params_of(s)
    cnt_w, lst = orc.neighbours(P, *s.pos.T)
    n = s.n
    img = [(row[: c] >= n).sum() for row, c in zip(lst, cnt_w)]
    img = np.array(img)
    z = s.pos[:, 2]
    # image j' of j is within 2h of i only if z_i + z_j < 2h: the lowest layers only
    assert (img[z > 2 * s.h] == 0).all()
    assert (img[z < 0.6 * s.dx] > 0).all()
