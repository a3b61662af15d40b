"""GPU parity of per-particle smoothing lengths (variable_h = 1) through the C-ABI against the FP64
oracle: neighbour counts, hash order, labels and dt bit for bit, state within 1e-12 (FP64) or 2e-5
(split) of each field's max-norm per step, on a body of two particle sizes with wall images, labels
and swaps, a dense case past the list capacity, and with the Heun and MUSCL variants."""
import numpy as np
import pytest

from oracle import orc
from paper_2310_03596_gb300 import gsph, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _err(g, o):
    scale = np.abs(o).max()
    return np.abs(g - o).max() / scale if scale > 0 else np.abs(g - o).max()


def _lockstep(scene, precision, steps, tol):
    P = orc.params_of(scene)
    sol = gsph.Solver.from_scene(scene, precision=precision, diagnostics=True)
    try:
        for k in range(steps):
            st = orc.OracleState.from_arrays(sol.state())
            do_swap = scene.K > 1 and scene.swap_period > 0 and k % scene.swap_period == 0
            dt_gpu = sol.dt()
            out = orc.step(P, st, do_swap=do_swap, want_rates=True)
            sol.step(1)
            sol.sync()
            assert dt_gpu == out["dt"], k
            assert np.array_equal(sol.get("hash"), out["key"])
            assert np.array_equal(sol.get("id"), st.id)
            assert np.array_equal(sol.get("label"), st.label)
            assert np.array_equal(sol.get("h"), st.h)
            assert np.array_equal(sol.get("nreal"), out["nreal"]), k
            assert np.array_equal(sol.get("nimage"), out["nimage"]), k
            stats = sol.exchange_stats()
            cost = np.bincount(st.label, weights=out["nreal"] + out["nimage"], minlength=scene.K)
            assert stats["cost"] == cost.astype(np.int64).tolist()
            for f in orc.FIELDS:
                e = _err(sol.get(f), getattr(st, f))
                assert e <= tol, (k, f, e)
    finally:
        sol.close()


PREC = [(gsph.FP64, 1e-12), (gsph.FP32_SPLIT, 2e-5)]


@pytest.mark.parametrize("precision,tol", PREC)
def test_two_sizes_lockstep(precision, tol):
    _lockstep(scenes.graded_block(seed=3), precision, 3, tol)                 # wall images
    _lockstep(scenes.graded_block(n_side=10, nz_fine=6, nz_coarse=4, seed=8, K=4), precision, 3, tol)
    s = scenes.graded_block(n_side=8, nz_fine=6, nz_coarse=4, seed=5, jitter=0.2)
    s.hp = 1.25 * s.hp                                                       # dense: past the list capacity
    s.h = float(s.hp.max())
    lo, dims = scenes._grid_around(s.pos, s.h, (4 * s.h,) * 3, (4 * s.h,) * 3)
    s.grid_lo, s.grid_dims = lo, dims
    _lockstep(s, precision, 2, tol)


@pytest.mark.parametrize("precision,tol", PREC)
def test_two_sizes_with_heun_and_muscl(precision, tol):
    s = scenes.graded_block(seed=11)
    s.integrator = 1
    _lockstep(s, precision, 2, tol)
    s = scenes.graded_block(seed=12)
    s.reconstruction = 1
    _lockstep(s, precision, 2, tol)


def test_equal_lengths_match_the_uniform_path():
    s = scenes.cube_impact(n_side=12, seed=2)
    a = gsph.Solver.from_scene(s, precision=gsph.FP64, diagnostics=True)
    s.variable_h = 1
    s.hp = np.full(s.n, s.h)
    b = gsph.Solver.from_scene(s, precision=gsph.FP64, diagnostics=True)
    try:
        # the time steps differ by the FP32 rounding of s_i / h_i: both take the uniform path's
        for _ in range(3):
            dt = a.dt()
            b.set_dt(dt)
            a.step(1)
            b.step(1)
        for f in ("nreal", "nimage", "hash", "id"):
            assert np.array_equal(a.get(f), b.get(f)), f
        for f in orc.FIELDS:
            assert _err(b.get(f), a.get(f)) <= 1e-13, f
    finally:
        a.close()
        b.close()


def test_variable_h_refusals():
    s = scenes.graded_block()
    with pytest.raises(gsph.GsphError) as ei:
        gsph.Solver.from_scene(s, overlap=True)
    assert ei.value.code == gsph.INVALID_ARG
    sol = gsph.Solver.from_scene(s, precision=gsph.FP64, diagnostics=True)
    try:
        for bad in (0.2 * s.h, 1.01 * s.h):
            with pytest.raises(gsph.GsphError) as ei:
                sol.put("h", np.full(s.n, bad))
            assert ei.value.code == gsph.INVALID_ARG
        import torch
        lam = torch.zeros((15, s.n), dtype=torch.float64, device="cuda")
        with pytest.raises(gsph.GsphError) as ei:
            sol.adjoint_step(lam, torch.empty_like(lam), 1e-9)
        assert ei.value.code == gsph.INVALID_ARG
    finally:
        sol.close()
