"""Pins of the oracle's communication hash / MGPU boundary set (Sec. II steps b-d) and the swap
heuristic (Sec. III.A, III.B)."""
import json
import math
import os

import numpy as np

from oracle import orc
from paper_2310_03596_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _decode(P, key):
    dx, dy = P.dims[0], P.dims[1]
    return np.stack([key % dx, (key // dx) % dy, key // (dx * dy)], 1).astype(np.int64)


def test_comm_hash_single_label_flags_nothing():
    s = scenes.cube_impact(n_side=10)
    P = orc.params_of(s)
    key = orc.hash_keys(P, *s.pos.T)
    flag, comm, cnt = orc.comm_hash(P, key, np.zeros(s.n, np.uint8))
    G = P.dims[0] * P.dims[1] * P.dims[2]
    assert flag.sum() == 0 and (comm == G).all() and cnt.sum() == 0


def test_comm_hash_brute_force_definition():
    # flagged iff a particle with another label lies in the same bucket or one of the 26 around it
    rng = np.random.default_rng(8)
    s = scenes.cube_impact(n_side=9, K=3, seed=8)
    P = orc.params_of(s)
    P.K = 3
    key = orc.hash_keys(P, *s.pos.T)
    G = P.dims[0] * P.dims[1] * P.dims[2]
    key[rng.choice(s.n, 5, replace=False)] = G     # a few garbage particles
    label = rng.integers(0, 3, s.n).astype(np.uint8)
    label[s.pos[:, 0] < 4e-3] = 0                   # a single-label region so both outcomes occur
    flag, comm, cnt = orc.comm_hash(P, key, label)
    c = _decode(P, key)
    want = np.zeros(s.n, np.uint8)
    for i in range(s.n):
        if key[i] == G:
            continue
        near = (np.abs(c - c[i]).max(axis=1) <= 1) & (key != G)
        want[i] = np.any(label[near] != label[i])
    assert np.array_equal(flag, want)
    assert 0 < want.sum() < s.n
    assert np.array_equal(comm, np.where(want == 1, key, G).astype(np.uint32))
    assert np.array_equal(cnt, np.bincount(label[want == 1], minlength=3))


def test_boundary_lists_are_the_comm_hash_sort_order():
    rng = np.random.default_rng(9)
    n, K, G = 2000, 4, 999
    label = rng.integers(0, K, n).astype(np.uint8)
    comm = np.where(rng.random(n) < 0.3, rng.integers(0, G, n), G).astype(np.uint32)
    off, out = orc.boundary_lists(label, comm, G, K)
    for k in range(K):
        mine = np.where(label == k)[0]
        order = mine[np.argsort(comm[mine], kind="stable")]
        want = order[comm[order] != G]
        assert np.array_equal(out[off[k]:off[k + 1]], want)


def test_cg_is_the_mean_to_the_fixed_point_quantum():
    s = scenes.taylor_bar(dx=1e-3, K=3)
    P = orc.params_of(s)
    step = np.array(s.grid_dims) * 2 * s.h / 2.0 ** 32      # the 32-bit fixed-point quantum
    for lab in range(3):
        cg, cnt = orc.cg(P, *s.pos.T, s.label, s.material, lab)
        sel = s.label == lab
        assert cnt == sel.sum()
        # each quantised coordinate lies within half a quantum (plus the FP64 rounding of the scaled
        # offset, 2^-20 quanta at most) of the position, so their mean does as well
        mean = np.array([np.mean(s.pos[sel][:, a].astype(np.longdouble)) for a in range(3)], dtype=np.float64)
        assert np.all(np.abs(cg - mean) <= step * (0.5 + 2.0 ** -19) + 4e-16 * np.abs(mean))


def test_cg_quantum_on_exact_grid_points():
    # a grid of extent 2^-4 at the origin: the quantum is 2^-36 and every position below is exact.
    # Multiples of the quantum give their own value back, half-way points tie to the even neighbour,
    # and positions outside the grid clamp to [0, 2^32 - 1] quanta
    s = scenes.taylor_bar(dx=1e-3, K=1)
    s.grid_lo, s.h, s.grid_dims = (0.0, 0.0, 0.0), 2.0 ** -8, (8, 8, 8)
    P = orc.params_of(s)
    q = 2.0 ** -36
    one = np.zeros(1, np.uint8)
    cases = [(0.0, 0), (q, 1), (7 * q, 7), ((2 ** 20 + 3) * q, 2 ** 20 + 3), (2.5 * q, 2), (3.5 * q, 4),
             ((2 ** 31 + 0.5) * q, 2 ** 31), ((2 ** 32 - 2) * q, 2 ** 32 - 2), (-1.0, 0), (1.0, 2 ** 32 - 1),
             (float("nan"), 0)]
    for xv, k in cases:
        cg, cnt = orc.cg(P, np.array([xv]), np.array([0.01]), np.array([0.01]), one, one, 0)
        assert cnt == 1 and cg[0] == k * q, (xv, k, cg[0] / q)
    # the sum of several is exact: the mean of 0, 1 and 2^32 - 2 quanta
    xs = np.array([0.0, q, (2 ** 32 - 2) * q])
    cg, _ = orc.cg(P, xs, np.full(3, 0.01), np.full(3, 0.01), np.zeros(3, np.uint8), np.zeros(3, np.uint8), 0)
    assert cg[0] == ((2 ** 32 - 1) / 3.0) * q


def test_balancing_hash_hand_worked():
    with open(os.path.join(GOLDEN, "balancing_hash_1d.json")) as f:
        g = json.load(f)
    for c in g["cases"]:
        assert orc.balancing_hash(g["own"], g["other"], c["p"]) == c["hash"], c
    for c in g["reverse_cases"]:
        assert orc.balancing_hash(g["other"], g["own"], c["p"]) == c["hash"], c
    # coincident Cgs: nothing to balance
    assert orc.balancing_hash([1.0, 1.0, 1.0], [1.0, 1.0, 1.0], [5.0, 0.0, 0.0]) == 0


def test_swap_two_labels_hand_worked():
    with open(os.path.join(GOLDEN, "swap_two_labels_1d.json")) as f:
        g = json.load(f)
    s = scenes.cube_impact(n_side=2)
    s.h, s.grid_lo, s.grid_dims, s.K = g["h"], tuple(g["grid_lo"]), tuple(g["grid_dims"]), 2
    P = orc.params_of(s)
    n = len(g["x"])
    st = orc.OracleState(n)
    st.x[:] = g["x"]
    st.label[:] = g["label_in"]
    cg0, _ = orc.cg(P, st.x, st.y, st.z, st.label, st.mat, 0)
    cg1, _ = orc.cg(P, st.x, st.y, st.z, st.label, st.mat, 1)
    h0 = [orc.balancing_hash(cg0, cg1, [x, 0, 0]) for x in st.x[:5]]
    h1 = [orc.balancing_hash(cg1, cg0, [x, 0, 0]) for x in st.x[5:]]
    assert h0 == g["hash_label0"] and h1 == g["hash_label1"]
    moved, pairs = orc.swap_pass(P, st)
    assert moved == 2 and pairs[0, 1] == 1
    assert st.label.tolist() == g["label_out"]


def test_swap_keeps_counts_and_shrinks_boundary_set():
    s = scenes.cube_impact(n_side=24, K=4, seed=12)
    P = orc.params_of(s)
    st = orc.OracleState.from_scene(s)
    key = orc.hash_keys(P, st.x, st.y, st.z)
    before = np.bincount(st.label, minlength=4)
    f0, _, _ = orc.comm_hash(P, key, st.label)
    fr = [f0.mean()]
    for _ in range(6):
        orc.swap_pass(P, st)
        assert np.array_equal(np.bincount(st.label, minlength=4), before)
        f, _, _ = orc.comm_hash(P, key, st.label)
        fr.append(f.mean())
    # from a random labelling almost every particle is on the MGPU boundary; the swaps pull each
    # label into a compact cloud (on this 24^3 cube with 2.6 dx buckets a 4-way split still flags
    # about 2/3 of the particles; the random labelling flags all of them)
    assert fr[0] > 0.95
    assert fr[-1] < 0.75 * fr[0]


def test_swap_per_type_keeps_label_type_counts():
    s = scenes.projectile_plate(dx=2e-3, radius=5e-3, plate=(30e-3, 30e-3, 6e-3), K=4)
    P = orc.params_of(s)
    st = orc.OracleState.from_scene(s)
    rng = np.random.default_rng(1)
    st.label[:] = rng.integers(0, 4, st.n)
    before = np.bincount(st.label.astype(int) * 2 + st.mat, minlength=8)
    moved, _ = orc.swap_pass(P, st)
    assert moved > 0
    assert np.array_equal(np.bincount(st.label.astype(int) * 2 + st.mat, minlength=8), before)


def test_swap_selection_by_brute_force_tiny():
    # for one label pair: the n highest-hash particles of each side (ties: lowest id) swap
    rng = np.random.default_rng(21)
    s = scenes.cube_impact(n_side=5, K=2, seed=21)
    P = orc.params_of(s)
    P.K = 2
    st = orc.OracleState.from_scene(s)
    st.label[:] = rng.integers(0, 2, st.n)
    st.id[:] = rng.permutation(st.n)
    lab0 = st.label.copy()
    cg0, _ = orc.cg(P, st.x, st.y, st.z, st.label, st.mat, 0)
    cg1, _ = orc.cg(P, st.x, st.y, st.z, st.label, st.mat, 1)
    P_ = np.stack([st.x, st.y, st.z], 1)
    h = np.array([orc.balancing_hash(cg0, cg1, p) if l == 0 else orc.balancing_hash(cg1, cg0, p)
                  for p, l in zip(P_, lab0)])
    a = [i for i in range(st.n) if lab0[i] == 0 and h[i] > 0]
    b = [i for i in range(st.n) if lab0[i] == 1 and h[i] > 0]
    m = min(len(a), len(b))
    assert m > 0
    pick = lambda idx: sorted(idx, key=lambda i: (-h[i], st.id[i]))[:m]
    want = lab0.copy()
    want[pick(a)] = 1
    want[pick(b)] = 0
    orc.swap_pass(P, st)
    assert np.array_equal(st.label, want)


def test_swap_two_types_biased_cg_hand_worked():
    # Sec. III.B's Cg' = alpha Cg_all + (1 - alpha) Cg_type, with Cg_all per label: a two-type,
    # two-label example whose outcome changes under the other readings (see the fixture)
    with open(os.path.join(GOLDEN, "swap_two_types_cg_prime.json")) as f:
        g = json.load(f)
    s = scenes.cube_impact(n_side=2)
    s.h, s.grid_lo, s.grid_dims, s.K, s.alpha = g["h"], tuple(g["grid_lo"]), tuple(g["grid_dims"]), 2, g["alpha"]
    s.materials = [s.materials[0], s.materials[0]]
    P = orc.params_of(s)
    assert P.nmat == 2
    n = len(g["x"])
    st = orc.OracleState(n)
    st.x[:] = g["x"]
    st.mat[:] = g["type"]
    st.label[:] = g["label_in"]
    st.id[:] = np.arange(n)
    moved, pairs = orc.swap_pass(P, st)
    assert moved == g["moved"] and pairs[0, 1] == 2
    assert st.label.tolist() == g["label_out"]
    assert g["label_out"] != g["label_out_other_readings"]


def _hash_fast_f32(M, d, dn, ell, p):
    """numpy float32 restatement of the swap kernel's FP32 fast path of the balancing hash: the hash
    from the FP32 roundings of the position and of the pair geometry, or -1 where the FP32 value with
    its error bound B (twice the first-order rounding bound plus 8 ulp) reaches a decision boundary."""
    f = np.float32
    Mf = np.array(M, dtype=np.float64).astype(f)
    u = (np.array(d) / dn).astype(f)
    scale = f(1000.0 / ell)
    pf = np.array(p, dtype=np.float64).astype(f)
    e = pf - Mf
    a = e * u
    t = (a[0] + a[1]) + a[2]
    v = f(t * scale)
    S = np.abs(a).sum(dtype=f)
    X = (np.abs(u) * (np.abs(pf) + np.abs(Mf))).sum(dtype=f)
    B = f(2.0 ** -23) * scale * (X + f(5) * S) + f(2.0 ** -21) * abs(v)
    lo, hi = f(v - B), f(v + B)
    if hi < 0:
        return 0
    if lo > 1000.5:
        return 1000
    if lo > 0 and hi < 999 and np.floor(lo) == np.floor(hi):
        k = int(np.floor(lo))
        return max(k, 1)
    return -1


def test_balancing_hash_fp32_fast_path_never_contradicts_fp64():
    # The swap kernel decides most balancing hashes from FP32 roundings and falls back to the FP64
    # definition within a rounding bound of a decision boundary. Positions placed within 1e-9 .. 1e-3
    # hash units of every kind of boundary (the middle, integer hashes, the other Cg), at Taylor-bar
    # scale coordinates: wherever the FP32 path decides, it equals the oracle's FP64 hash.
    rng = np.random.default_rng(44)
    decided = total = 0
    mid_decided = mid_total = 0
    for trial in range(60):
        ca = rng.uniform(-5e-3, 40e-3, 3)
        cb = ca + rng.normal(0, 10.0 ** rng.uniform(-6, -2), 3)
        M = (ca + cb) * 0.5
        d = cb - ca
        dn = math.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
        ell = dn * 0.5
        n = d / dn
        perp = np.cross(n, rng.normal(size=3))
        for k in (0, 1, 2, 250, 998, 999, 1000):
            for delta in (-1e-3, -1e-6, -1e-9, 0.0, 1e-9, 1e-6, 1e-3, 0.37):
                V = k + delta
                p = M + (V / 1000.0 * ell) * n + rng.uniform(-2e-3, 2e-3) * perp
                want = orc.balancing_hash(ca, cb, p)
                got = _hash_fast_f32(M, d, dn, ell, p)
                total += 1
                if got >= 0:
                    decided += 1
                    assert got == want, (trial, k, delta, got, want)
                if delta == 0.37 and k < 999 and ell > 2e-4:
                    mid_total += 1
                    mid_decided += got >= 0
    # away from the boundaries (mid-interval, Cgs more than 0.4 mm apart) FP32 decides
    assert decided > 0 and mid_total > 30 and mid_decided == mid_total
