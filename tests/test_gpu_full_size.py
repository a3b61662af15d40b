"""Full-size parity in the benchmark's launch configuration (Taylor bar, 1,607,680 particles, FP32
split, K = 4 labels, swap heuristic and communication hash every step, diagnostics off).

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


def test_taylor_bar_full_size_step():
    s = scenes.taylor_bar()
    P = orc.params_of(s)
    sol = gsph.Solver.from_scene(s, precision=gsph.FP32_SPLIT)
    sol.step(3)                                     # the impact has started
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
    # swap pass (step index 3, period 1) and communication hash on the sorted view
    moved, _ = orc.swap_pass(P, st)
    assert np.array_equal(sol.get("label"), st.label)
    flag, comm, cnt = orc.comm_hash(P, skey, st.label)
    assert np.array_equal(sol.get("flag"), flag)
    assert np.array_equal(sol.get("comm_hash"), comm)
    stats = sol.exchange_stats()
    assert stats["boundary"] == cnt.tolist()
    assert stats["swapped_last_pass"] == moved
    # sampled interaction + integration
    rng = np.random.default_rng(17)
    sample = np.sort(rng.choice(s.n, 3000, replace=False))
    # include particles in contact with the wall, where the flow is non-trivial
    low = np.where(st.z < 2 * s.h)[0]
    sample = np.unique(np.concatenate([sample, rng.choice(low, 500, replace=False)]))
    r, nr, ni = orc.rates(P, st, subset=sample)
    sub = orc.OracleState.from_arrays({k: v[sample] for k, v in st.arrays().items()})
    orc.integrate(P, sub, r[sample], dt)
    g = sol.state()
    for f in STATE:
        gv, ov = g[f][sample], getattr(sub, f)
        scale = max(np.abs(getattr(st, f)).max(), np.abs(ov).max(), 1e-300)
        assert np.abs(gv - ov).max() <= 2e-5 * scale, f


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
