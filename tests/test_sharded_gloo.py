"""The label-sharded data plane (paper_2310_03596_gb300.sharded) on 2 and 4 gloo ranks on CPU, one
ownership label per rank, against the single-device run with K virtual labels. Each rank's interaction
engine here is the FP64 oracle (the CPU stand-in for the GPU engine); the exchanges are the real
collectives: the allreduce (bitwise OR) of the bucket label masks, the allgatherv of the MGPU boundary
records into the halo, the swap pass's sums and the exchange of the swapped particles. Hashes, flags,
boundary counts, neighbour counts, labels and dt match bit for bit; the FP64 state within 1e-12."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleEngine:
    """Interaction + integration of a rank's own particles (the first n_own of the union) by the
    oracle, over its own and halo particles."""

    def __init__(self, P):
        self.P = P

    def _state(self, st, n=None):
        from oracle import orc
        d = {f: st[f][:n].numpy() if n is not None else st[f].numpy() for f in st}
        return orc.OracleState.from_arrays({**d, "material": d["mat"], "id": d["id"].astype(np.uint32)})

    def advance(self, union, n_own, dt):
        from oracle import orc
        from paper_2310_03596_gb300.sharded import STATE
        u = self._state(union)
        r, nr, ni = orc.rates(self.P, u, subset=np.arange(n_own))
        own = self._state(union, n_own)
        orc.integrate(self.P, own, r[:n_own], dt)
        new = {f: torch.from_numpy(np.array(getattr(own, f))) for f in STATE}
        for f in ("mat", "label", "id"):
            new[f] = union[f][:n_own].clone()
        return new, torch.from_numpy(nr[:n_own].copy()), torch.from_numpy(ni[:n_own].copy())

    def dt(self, st):
        from oracle import orc
        return orc.dt(self.P, self._state(st))


def _scene(kind, K):
    from paper_2310_03596_gb300 import scenes
    if kind == "cube":
        s = scenes.cube_impact(n_side=9, K=K, seed=17)
        s.swap_period = 2
    else:   # two materials: per-type swaps with the biased Cg' (Sec. III.B)
        s = scenes.projectile_plate(dx=2e-3, radius=4e-3, plate=(24e-3, 24e-3, 6e-3), K=K)
        rng = np.random.default_rng(5)
        s.label = rng.integers(0, K, s.n).astype(np.uint8)
        s.swap_period = 1
    return s


def _rank(rank, world, port, kind, steps, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import orc
        from paper_2310_03596_gb300 import sharded
        s = _scene(kind, world)
        P = orc.params_of(s)
        sol = sharded.ShardedSolver(s, OracleEngine(P))
        per_step = []
        for _ in range(steps):
            sol.step()
            L = sol.last
            parts = [None] * world
            dist.all_gather_object(parts, {k: (v.numpy() if torch.is_tensor(v) else v) for k, v in L.items()})
            per_step.append(parts)
        final = sol.gather()
        if rank == 0:
            q.put(("ok", per_step, final))
    except Exception as e:   # noqa: BLE001
        q.put(("error", repr(e), None))
        raise
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,kind", [(2, "cube"), (4, "cube"), (2, "plate")])
def test_sharded_run_matches_single_device(world, kind):
    import sys
    sys.path.insert(0, ROOT)
    from oracle import orc
    orc.build()
    steps = 4
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, kind, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    status, per_step, final = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
    assert status == "ok", per_step
    assert all(p.exitcode == 0 for p in procs)
    # the single-device run with K virtual labels
    s = _scene(kind, world)
    P = orc.params_of(s)
    st = orc.OracleState.from_scene(s)
    swaps = 0
    for k in range(steps):
        out = orc.step(P, st, do_swap=(k % s.swap_period == 0))
        parts = per_step[k]
        ids = np.concatenate([p["id"] for p in parts])
        o = np.argsort(ids)
        so = np.argsort(st.id)
        for name, want in (("key", out["key"]), ("flag", out["flag"]), ("nreal", out["nreal"]),
                           ("nimage", out["nimage"])):
            got = np.concatenate([p[name] for p in parts])[o]
            assert np.array_equal(got.astype(np.int64), np.asarray(want)[so].astype(np.int64)), (k, name)
        assert np.array_equal(parts[0]["counts"], out["count"]), k
        assert all(p["dt"] == out["dt"] for p in parts), k
        lab = np.concatenate([np.full(len(p["id"]), r) for r, p in enumerate(parts)])[o]
        assert np.array_equal(lab, st.label[so]), k          # ownership = the label after the swap pass
        swaps += parts[0]["moved"]
    # final state, labels and every field
    so = np.argsort(st.id)
    assert np.array_equal(final["id"], st.id[so].astype(np.int64))
    assert np.array_equal(final["label"], st.label[so])
    for f in orc.FIELDS:
        want = getattr(st, f)[so]
        scale = max(np.abs(want).max(), 1e-300)
        assert np.abs(final[f] - want).max() <= 1e-12 * scale, f
    assert swaps > 0
    halos = [p["halo"] for parts in per_step for p in parts]
    assert min(halos) > 0          # every rank received boundary records at every step
    print(kind, world, "halo sizes", halos, "moved", swaps)


def _rank_leaves(rank, world, port, q):
    import datetime
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    from paper_2310_03596_gb300 import scenes, sharded
    from oracle import orc
    s = _scene("cube", world)
    sol = sharded.ShardedSolver(s, OracleEngine(orc.params_of(s)))
    sol.step()
    if rank == world - 1:
        q.put((rank, "left"))       # this rank leaves between steps, with no collective in flight
        q.close()
        q.join_thread()
        os._exit(0)
    try:
        sol.step()                  # the next step's collectives cannot complete
        q.put((rank, "no error"))
    except Exception as e:          # noqa: BLE001
        q.put((rank, type(e).__name__))
    q.close()
    q.join_thread()
    os._exit(0)


def test_a_rank_that_leaves_ends_the_others_next_step_with_an_error():
    # failure detection on the host: the remaining ranks' next collective ends with an error within
    # the process group's timeout instead of waiting forever
    import time
    from oracle import orc
    orc.build()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    t0 = time.time()
    procs = [ctx.Process(target=_rank_leaves, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
    assert got[world - 1] == "left"
    assert got[0] != "no error", got
    assert time.time() - t0 < 110
