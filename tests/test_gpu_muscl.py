"""GPU parity of the MUSCL reconstruction (reconstruction = 1) through the C-ABI against the FP64
oracle: the gradient pass and the reconstructed fluxes, with wall images (mirrored states and
gradients), labels and swaps, and neighbours beyond the list capacity (re-scan path). Integer and
order outputs bit for bit; state within 1e-12 (FP64) or 2e-5 (split) of each field's max-norm per
step, and the step's rates (diagnostics) within 1e-11 (FP64) or 1e-4 (split)."""
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


def _lockstep_muscl(scene, precision, steps, tol, rtol):
    scene.reconstruction = 1
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
            assert dt_gpu == out["dt"]
            assert np.array_equal(sol.get("hash"), out["key"])
            assert np.array_equal(sol.get("id"), st.id)
            assert np.array_equal(sol.get("label"), st.label)
            assert np.array_equal(sol.get("nreal"), out["nreal"])
            assert np.array_equal(sol.get("nimage"), out["nimage"])
            gr = sol.get("rates")
            for c in range(orc.NRATE):
                e = _err(gr[:, c], out["rates"][:, c])
                assert e <= rtol, (k, "rate", c, e)
            for f in orc.FIELDS:
                e = _err(sol.get(f), getattr(st, f))
                assert e <= tol, (k, f, e)
    finally:
        sol.close()


@pytest.mark.parametrize("precision,tol,rtol", [(gsph.FP64, 1e-12, 1e-11), (gsph.FP32_SPLIT, 2e-5, 1e-4)])
def test_muscl_lockstep(precision, tol, rtol):
    # wall images (cube impact), labels and swaps (Taylor bar), list overflow (dense)
    _lockstep_muscl(scenes.cube_impact(n_side=12, seed=17), precision, 3, tol, rtol)
    _lockstep_muscl(scenes.taylor_bar(dx=0.5e-3, K=4, swap_period=1), precision, 2, tol, rtol)
    s = scenes.cube_impact(n_side=10, seed=9)
    s.h = 1.6 * s.dx
    lo = tuple(v - 4 * s.h for v in s.pos.min(axis=0))
    s.grid_lo = lo
    s.grid_dims = tuple(int(np.ceil((s.pos[:, a].max() + 4 * s.h - lo[a]) / (2 * s.h))) for a in range(3))
    _lockstep_muscl(s, precision, 2, tol, rtol)


@pytest.mark.parametrize("precision,bound", [(gsph.FP64, 1e-13), (gsph.FP32_SPLIT, 1e-6)])
def test_muscl_fluxes_conserve_on_a_free_body(precision, bound):
    s = scenes.cube_impact(n_side=12, seed=3)
    s.walls = []
    s.reconstruction = 1
    rng = np.random.default_rng(4)
    X = s.pos
    s.vel = np.stack([20.0 * np.sin(800.0 * X[:, 1]), 10.0 * np.cos(600.0 * X[:, 2]),
                      30.0 * np.sin(700.0 * X[:, 0])], 1) + rng.normal(0, 2.0, X.shape)
    sol = gsph.Solver.from_scene(s, precision=precision, diagnostics=True)
    try:
        sol.step(2)          # stresses and densities develop from the velocity field
        sol.sync()
        r = sol.get("rates")
        for c in (1, 2, 3, 4, 5):
            assert abs(r[:, c].sum()) <= bound * np.abs(r[:, c]).sum(), c
    finally:
        sol.close()


def test_muscl_refuses_heun_overlap_and_adjoint():
    s = scenes.cube_impact(n_side=6)
    s.reconstruction = 1
    s.integrator = 1
    with pytest.raises(gsph.GsphError) as ei:
        gsph.Solver.from_scene(s)
    assert ei.value.code == gsph.INVALID_ARG
    s.integrator = 0
    with pytest.raises(gsph.GsphError) as ei:
        gsph.Solver.from_scene(s, overlap=True)
    assert ei.value.code == gsph.INVALID_ARG
    sol = gsph.Solver.from_scene(s, precision=gsph.FP64, diagnostics=True)
    try:
        import torch
        lam = torch.zeros((15, s.n), dtype=torch.float64, device="cuda")
        with pytest.raises(gsph.GsphError) as ei:
            sol.adjoint_step(lam, torch.empty_like(lam), 1e-9)
        assert ei.value.code == gsph.INVALID_ARG
    finally:
        sol.close()
