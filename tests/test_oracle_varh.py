"""Pins of the variable smoothing-length reading (Sec. V's varying particle sizes): per-particle h_i,
pair smoothing length h_ij = (h_i + h_j) / 2, support r^2 < (h_i + h_j)^2, buckets of side 2 h_max,
dt = cfl min_i h_i / s_i.

- the bucket search finds exactly the brute-force neighbour sets of the per-pair supports;
- h_i = h everywhere reproduces the uniform-h rates bit for bit;
- the pair terms stay antisymmetric (h_ij is symmetric): mass, momentum and energy are conserved on a
  free body of two particle sizes, and a two-particle pair is bitwise antisymmetric;
- the velocity gradient of a linear field is A M in the interior of both resolutions, M the lattice
  moment at h / dx = 1.3 (summed here independently of the oracle): the kernel takes each pair's own h;
- at rest and uniform density the time step is cfl h_min / c.
"""
import numpy as np
import pytest

from oracle import orc
from paper_2310_03596_gb300 import scenes


def _block(**kw):
    s = scenes.graded_block(**kw)
    return s, orc.params_of(s), orc.OracleState.from_scene(s)


def test_bucket_search_matches_brute_force_with_per_pair_supports():
    rng = np.random.default_rng(2)
    s, P, st = _block(jitter=0.3, seed=4)
    h = st.h.copy()
    h[rng.random(st.n) < 0.3] *= 0.77          # three sizes, random
    cb, lb = orc.neighbours(P, st.x, st.y, st.z, cap=700, brute=True, h=h)
    cc, lc = orc.neighbours(P, st.x, st.y, st.z, cap=700, h=h)
    assert np.array_equal(cb, cc)
    assert np.array_equal(np.sort(lb, axis=1), np.sort(lc, axis=1))
    assert (cb > 0).all() and cb.max() > 2 * np.median(cb)   # coarse particles see many fine ones


def test_uniform_lengths_reproduce_the_uniform_rates_bitwise():
    s = scenes.cube_impact(n_side=8, seed=5)
    P0 = orc.params_of(s)
    st = orc.OracleState.from_scene(s)
    st.vx[:] = np.random.default_rng(1).normal(0, 5.0, st.n)
    r0, n0, i0 = orc.rates(P0, st)
    s.variable_h = 1
    P1 = orc.params_of(s)
    st.h = np.full(st.n, s.h)
    r1, n1, i1 = orc.rates(P1, st)
    assert np.array_equal(n0, n1) and np.array_equal(i0, i1)
    assert np.array_equal(r0, r1)


def test_two_sizes_pair_is_bitwise_antisymmetric_and_body_conserves():
    s, P, st = _block(n_side=4, nz_fine=2, nz_coarse=2, wall=False)
    # the lowest coarse particle and a fine particle below it
    ic = int(np.argmin(np.where(st.h > st.h.min(), st.z, np.inf)))
    d = np.hypot(np.hypot(st.x - st.x[ic], st.y - st.y[ic]), st.z - st.z[ic])
    jf = int(np.argmin(np.where(st.h == st.h.min(), d, np.inf)))
    two = orc.OracleState.from_arrays({k: v[[jf, ic]] for k, v in st.arrays().items()})
    two.vx[:] = [30.0, -10.0]; two.vz[:] = [-3.0, 4.0]
    two.sxy[:] = [1e7, -3e7]; two.sxx[:] = [2e7, 0.0]; two.syy[:] = [-2e7, 0.0]; two.szz[:] = [0.0, 0.0]
    r, nr, _ = orc.rates(P, two)
    assert nr.tolist() == [1, 1]
    for k in (1, 2, 3, 4, 5):
        assert r[0, k] == -r[1, k], k
    # a free body of both sizes with a random state
    s, P, st = _block(n_side=8, nz_fine=6, nz_coarse=4, jitter=0.05, wall=False)
    rng = np.random.default_rng(3)
    for f in ("vx", "vy", "vz"):
        getattr(st, f)[:] = rng.normal(0, 5.0, st.n)
    for f in ("sxx", "syy", "sxy", "sxz", "syz"):
        getattr(st, f)[:] = rng.normal(0, 3e7, st.n)
    st.szz[:] = -(st.sxx + st.syy)
    st.m[:] *= 1 + 0.01 * rng.standard_normal(st.n)
    r, _, _ = orc.rates(P, st)
    for k in (1, 2, 3, 4, 5):
        assert abs(r[:, k].sum()) <= 1e-13 * np.abs(r[:, k]).sum(), k


def _lattice_moment(ratio):
    m = int(np.ceil(2 * ratio))
    M = np.zeros((3, 3))
    for i in range(-m, m + 1):
        for j in range(-m, m + 1):
            for k in range(-m, m + 1):
                d = np.array([i, j, k], float)
                r = np.sqrt(d @ d)
                if r == 0 or not r < 2 * ratio:
                    continue
                M += np.outer(d, orc.kernel_dw(r, ratio) * d / r)
    return M


def test_velocity_gradient_uses_each_pairs_smoothing_length():
    s, P, st = _block(n_side=16, nz_fine=12, nz_coarse=12, jitter=0.0, wall=False)
    A = np.array([[0.0, 300.0, 0.0], [0.0, 0.0, 50.0], [100.0, 0.0, -200.0]])
    X = np.stack([st.x, st.y, st.z], 1)
    V = X @ A.T
    st.vx[:], st.vy[:], st.vz[:] = V[:, 0], V[:, 1], V[:, 2]
    r, _, _ = orc.rates(P, st)
    L = r[:, 6:15].reshape(-1, 3, 3)
    M = _lattice_moment(1.3)               # unit spacing, h = 1.3: the moment at h / dx = 1.3
    exp = A @ M
    hf, hc = st.h.min(), st.h.max()
    zf = 12 * s.dx
    x0, x1 = st.x.min(), st.x.max()
    for fine, lo, hi, hh in ((True, 2 * hc, zf - 2 * hc, hf), (False, zf + 2 * hc, st.z.max() - 2 * hc, hc)):
        sel = (st.h == hh) & (st.z > lo) & (st.z < hi)
        for a, b in ((st.x, (x0, x1)), (st.y, (st.y.min(), st.y.max()))):
            sel &= (a > b[0] + 2 * hc) & (a < b[1] - 2 * hc)
        assert sel.sum() > 0, fine
        assert np.abs(L[sel] - exp).max() <= 1e-9 * np.abs(exp).max(), fine


def test_time_step_at_rest_is_cfl_hmin_over_c():
    s, P, st = _block()
    st.vx[:] = 0.0; st.vy[:] = 0.0; st.vz[:] = 0.0; st.E[:] = 0.0
    rho0, K, G, _ = s.materials[0]
    c = np.sqrt((K + 4 * G / 3) / rho0)
    dt = orc.dt(P, st)
    assert dt == pytest.approx(s.cfl * st.h.min() / c, rel=1e-15)
