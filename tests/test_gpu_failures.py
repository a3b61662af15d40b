"""Failure detection without a GPU fault: the swap pass's bounded grid barrier is made to run out (it
waits for one block more than it launched, with a short limit), and a device allocation is made to fail
on the host. Each returns its status and leaves the context usable."""
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


def test_swap_barrier_timeout_is_reported_and_the_next_pass_succeeds():
    s = scenes.cube_impact(n_side=10, K=4, seed=2)
    s.swap_period = 1
    sol = gsph.Solver.from_scene(s, precision=gsph.FP64, diagnostics=True)
    lab0 = sol.get("label")
    L = sol.L
    assert L.gsph_set_wait_limit(sol.h, 64, 1) == gsph.OK
    sol.swap_now()
    assert L.gsph_sync(sol.h, None) == gsph.DEVICE_TIMEOUT
    # the pass gave up at its first barrier: no label changed
    assert np.array_equal(sol.get("label"), lab0)
    # restored limits: the next pass on the same context matches the oracle again
    assert L.gsph_set_wait_limit(sol.h, 0, 0) == gsph.OK
    st = orc.OracleState.from_arrays(sol.state())
    out = orc.step(orc.params_of(s), st, do_swap=True)
    sol.step(1)
    sol.sync()
    assert np.array_equal(sol.get("label"), st.label)
    assert np.array_equal(sol.get("id"), st.id)
    assert sol.dt() == orc.dt(orc.params_of(s), st)
    del out
    sol.close()


def test_failed_allocation_returns_oom_and_keeps_the_particles():
    s = scenes.cube_impact(n_side=8, K=2, seed=3)
    sol = gsph.Solver.from_scene(s, precision=gsph.FP32_SPLIT)
    sol.step(2)
    sol.sync()
    before = sol.state()
    big = scenes.cube_impact(n_side=12, K=2, seed=3)
    for k in (1, 7, 30):      # the first, an intermediate and a late allocation of the new set
        gsph.load().gsph_debug_fail_alloc(k)
        with pytest.raises(gsph.GsphError) as ei:
            sol.set_particles(big.pos, big.vel, big.vol, big.material, big.label)
        assert ei.value.code == gsph.OOM
        gsph.load().gsph_debug_fail_alloc(0)
        assert sol.sizes()[0] == s.n
        after = sol.state()
        for f in STATE + ("id", "label"):
            assert np.array_equal(after[f], before[f]), (k, f)
    # the context keeps stepping, and takes the bigger set once allocation works again
    sol.step(1)
    sol.sync()
    sol.set_particles(big.pos, big.vel, big.vol, big.material, big.label)
    sol.step(1)
    sol.sync()
    assert sol.sizes()[0] == big.n
    sol.close()
