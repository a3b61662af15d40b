"""Steps enqueued by one gsph_step call run partly concurrently: the communication hash beside the
neighbour-list build, and each step's time-step reduction beside the next step's hash, sort and
reorder, on a second stream of the context. These tests check, through the C-ABI, that n steps in one
call give the same bits as n calls of one step (state, labels, hash, flags, dt, pair count), on both
precisions, with the swap pass every step or every other step, and in the two-pass interaction order."""
import numpy as np
import pytest

from oracle import orc
from paper_2310_03596_gb300 import gsph, scenes

pytestmark = pytest.mark.gpu

FIELDS = list(orc.FIELDS) + ["id", "label", "material", "hash", "comm_hash", "flag"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _same_after(scene, precision, steps, overlap=False):
    batched = gsph.Solver.from_scene(scene, precision=precision, overlap=overlap)
    single = gsph.Solver.from_scene(scene, precision=precision, overlap=overlap)
    try:
        batched.step(steps)
        for _ in range(steps):
            single.step(1)
        batched.sync()
        single.sync()
        assert batched.dt() == single.dt()
        for f in FIELDS:
            assert np.array_equal(batched.get(f), single.get(f)), f
        sb, ss = batched.exchange_stats(), single.exchange_stats()
        assert sb["pairs_total"] == ss["pairs_total"]
        assert sb["swap_passes"] == ss["swap_passes"] > 0
    finally:
        batched.close()
        single.close()


@pytest.mark.parametrize("precision", [gsph.FP32_SPLIT, gsph.FP64])
def test_one_call_of_n_steps_equals_n_calls(precision):
    s = scenes.taylor_bar(dx=0.5e-3, K=4, swap_period=1)
    _same_after(s, precision, 7)


def test_one_call_equals_n_calls_sixteen_labels_every_other_step():
    s = scenes.collapse_block(dx=4e-3, size=(0.12, 0.06, 0.04), K=16, swap_period=2)
    _same_after(s, gsph.FP32_SPLIT, 6)


def test_one_call_equals_n_calls_two_pass_order():
    s = scenes.taylor_bar(dx=0.5e-3, K=4, swap_period=1)
    _same_after(s, gsph.FP32_SPLIT, 5, overlap=True)


@pytest.mark.parametrize("overlap", [False, True])
def test_timing_scopes_leave_the_state_alone(overlap):
    """Phase events (every phase, or only those that bound the pair kernel) change no bit of the state;
    the pair-only scope fills pair_ms alone, and its pair time agrees with the full scope's."""
    s = scenes.taylor_bar(dx=0.5e-3, K=4, swap_period=1)
    sols = {k: gsph.Solver.from_scene(s, overlap=overlap) for k in ("none", "all", "pair")}
    try:
        sols["all"].set_timing(6)
        sols["pair"].set_timing(6, pair_only=True)
        for sol in sols.values():
            sol.step(6)
            sol.sync()
        for f in FIELDS:
            assert np.array_equal(sols["none"].get(f), sols["all"].get(f)), f
            assert np.array_equal(sols["none"].get(f), sols["pair"].get(f)), f
        ta, tp = sols["all"].timings(), sols["pair"].timings()
        assert ta["steps"] == tp["steps"] == 6
        assert ta["hash_sort_ms"] > 0 and ta["nbr_list_ms"] > 0 and ta["pair_ms"] > 0
        assert tp["pair_ms"] > 0
        assert all(v == 0 for k, v in tp.items() if k.endswith("_ms") and k != "pair_ms")
        assert 0.5 < tp["pair_ms"] / ta["pair_ms"] < 2.0
    finally:
        for sol in sols.values():
            sol.close()
