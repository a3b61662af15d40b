"""Full-size parity in the benchmark's launch configuration (FP32 split, diagnostics off) on the Taylor
bar (1,607,680 particles, K = 4, swap and communication hash every step), the projectile on the plate
(4,565,752 particles, two materials, K = 8) and the collapse block (64,000,000 particles, K = 16), and
the bench's variant lines at their sizes (the FP64 path, MUSCL, the two-resolution bar).

Integer outputs are compared on every particle; the new floating-point state on a random sample of
particles whose rates and integration the oracle computes one by one.
"""
import json
import os

import numpy as np
import pytest

from oracle import orc
from paper_2310_03596_gb300 import gsph, scenes

pytestmark = pytest.mark.gpu
STATE = tuple(gsph.FIELDS[:15])


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _full_size_step(s, before, nsample=3000, seed=17, precision=gsph.FP32_SPLIT, tol=2e-5):
    """`before` steps on the GPU, then one step compared with the oracle: hash, sort, swap pass (when
    the step index is a multiple of the period), communication hash on every particle; the rates and
    integration of a sample (plus particles in wall contact) one by one."""
    P = orc.params_of(s)
    sol = gsph.Solver.from_scene(s, precision=precision)
    try:
        sol.step(before)
        st = orc.OracleState.from_arrays(sol.state())
        dt = sol.dt()
        sol.step(1)
        sol.sync()
        # oracle: hash and stable sort of the whole set
        key = orc.hash_keys(P, st.x, st.y, st.z)
        perm = orc.sort_order(key)
        st.permute(perm)
        skey = key[perm]
        assert np.array_equal(sol.get("hash"), skey)
        assert np.array_equal(sol.get("id"), st.id)
        stats = sol.exchange_stats()
        if s.K > 1 and s.swap_period > 0 and before % s.swap_period == 0:
            moved, _ = orc.swap_pass(P, st)
            assert stats["swapped_last_pass"] == moved
        assert np.array_equal(sol.get("label"), st.label)
        flag, comm, cnt = orc.comm_hash(P, skey, st.label)
        assert np.array_equal(sol.get("flag"), flag)
        assert np.array_equal(sol.get("comm_hash"), comm)
        assert stats["boundary"] == cnt.tolist()
        # sampled interaction + integration
        rng = np.random.default_rng(seed)
        sample = np.sort(rng.choice(s.n, nsample, replace=False))
        # include particles in contact with the wall, where the flow is non-trivial
        low = np.where(st.z < 2 * s.h)[0] if s.walls else np.zeros(0, np.int64)
        if len(low):
            sample = np.unique(np.concatenate([sample, rng.choice(low, min(500, len(low)), replace=False)]))
        r, nr, ni = orc.rates(P, st, subset=sample)
        sub = orc.OracleState.from_arrays({k: v[sample] for k, v in st.arrays().items()})
        orc.integrate(P, sub, r[sample], dt)
        g = sol.state()
        # a vector or tensor component is measured against the max-norm of its field (v, S): at the
        # first step of a body at rest in x and y those components are rounding noise
        group = {f: ("vx", "vy", "vz") for f in ("vx", "vy", "vz")}
        group.update({f: ("sxx", "syy", "szz", "sxy", "sxz", "syz") for f in ("sxx", "syy", "szz", "sxy", "sxz", "syz")})
        for f in STATE:
            gv, ov = g[f][sample], getattr(sub, f)
            scale = max(max(np.abs(getattr(st, c)).max() for c in group.get(f, (f,))), np.abs(ov).max(), 1e-300)
            assert np.abs(gv - ov).max() <= tol * scale, f
    finally:
        sol.close()


def test_taylor_bar_full_size_step():
    # 1,607,680 particles, K = 4, swaps every step; step 3: the impact has started
    _full_size_step(scenes.taylor_bar(), 3)


def test_taylor_bar_full_size_fp64_step():
    # the FP64 path at full size: 1e-12 of each field's max-norm
    _full_size_step(scenes.taylor_bar(), 2, seed=21, precision=gsph.FP64, tol=1e-12)


def test_taylor_bar_full_size_muscl_step():
    # the bench's MUSCL line: gradient pass and reconstructed fluxes at full size
    s = scenes.taylor_bar()
    s.reconstruction = 1
    _full_size_step(s, 3, seed=22)


def test_graded_bar_full_size_step():
    # the bench's varying-size line: 553,600 particles of two sizes
    _full_size_step(scenes.graded_bar(), 3, seed=23)


def test_projectile_plate_full_size_step():
    # 4,565,752 particles of two materials, K = 8 slabs; step 0 runs the per-type swap pass
    _full_size_step(scenes.projectile_plate(), 0, seed=18)


def test_collapse_block_full_size_step():
    # 64,000,000 particles under gravity on the floor, K = 16; step 0 runs the swap pass (120 pairs)
    _full_size_step(scenes.collapse_block(), 0, nsample=2000, seed=19)


def test_split_path_error_report():
    """Per-field error of the FP32-split path against the FP64 oracle on the cube impact: rates of one
    step (lockstep) and the state after 1 and after 100 free steps, each relative to the field's
    max-norm. Written to $GSPH_ERROR_REPORT when set."""
    s = scenes.cube_impact(n_side=16, steps=100)
    P = orc.params_of(s)
    report = {"rates_1_step": {}, "state_1_step": {}, "state_100_steps": {}}
    sol = gsph.Solver.from_scene(s, precision=gsph.FP32_SPLIT, diagnostics=True)
    sol.step(5)
    st = orc.OracleState.from_arrays(sol.state())
    out = orc.step(P, st, want_rates=True)
    sol.step(1)
    gr = sol.get("rates")
    names = ["dw", "dm", "dmvx", "dmvy", "dmvz", "dmE"] + [f"L{u}{v}" for u in "xyz" for v in "xyz"]
    for k, name in enumerate(names):
        o = out["rates"][:, k]
        report["rates_1_step"][name] = float(np.abs(gr[:, k] - o).max() / max(np.abs(o).max(), 1e-300))
    for f in STATE:
        o = getattr(st, f)
        report["state_1_step"][f] = float(np.abs(sol.get(f) - o).max() / max(np.abs(o).max(), 1e-300))
    sol.close()
    # free running, 100 steps from the initial state
    st = orc.OracleState.from_scene(s)
    for _ in range(100):
        orc.step(P, st)
    sol = gsph.Solver.from_scene(s, precision=gsph.FP32_SPLIT)
    sol.step(100)
    g = sol.state()
    order = np.argsort(g["id"])
    ref = np.argsort(st.id)
    for f in STATE:
        o = getattr(st, f)[ref]
        report["state_100_steps"][f] = float(np.abs(g[f][order] - o).max() / max(np.abs(o).max(), 1e-300))
    sol.close()
    path = os.environ.get("GSPH_ERROR_REPORT")
    if path:
        with open(path, "w") as fh:
            json.dump(report, fh, indent=1)
    assert max(report["rates_1_step"].values()) < 1e-4
    assert max(report["state_1_step"].values()) < 2e-5
    assert max(report["state_100_steps"].values()) < 1e-3
