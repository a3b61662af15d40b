"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle on the same seeded inputs.

Integer, index and order outputs (bucket hash, sort order, neighbour counts, flags, communication
hash, boundary set, labels after swaps, dt) must match bit for bit. FP64 state must match within
1e-12 of each field's max-norm per step; the split path within 2e-5 per step and 1e-3 after 100 free
steps (the stated tolerances, relative to the field's max-norm over particles).
"""
import numpy as np
import pytest

from oracle import orc
from paper_2310_03596_gb300 import gsph, scenes

pytestmark = pytest.mark.gpu

STATE_F = orc.FIELDS


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _maxnorm_err(g, o):
    scale = np.abs(o).max()
    return np.abs(g - o).max() / scale if scale > 0 else np.abs(g - o).max()


def _lockstep(scene, precision, steps, tol, swap=True, overlap=False):
    P = orc.params_of(scene)
    sol = gsph.Solver.from_scene(scene, precision=precision, diagnostics=True, overlap=overlap)
    worst = {f: 0.0 for f in STATE_F}
    try:
        for k in range(steps):
            st = orc.OracleState.from_arrays(sol.state())
            do_swap = swap and scene.K > 1 and scene.swap_period > 0 and k % scene.swap_period == 0
            dt_gpu = sol.dt()
            out = orc.step(P, st, do_swap=do_swap, want_rates=True)
            sol.step(1)
            sol.sync()
            assert dt_gpu == out["dt"]
            assert np.array_equal(sol.get("hash"), out["key"]), "hash / sort order"
            assert np.array_equal(sol.get("id"), st.id), "sort order"
            assert np.array_equal(sol.get("label"), st.label), "labels"
            assert np.array_equal(sol.get("material"), st.mat)
            assert np.array_equal(sol.get("nreal"), out["nreal"]), "real neighbour counts"
            assert np.array_equal(sol.get("nimage"), out["nimage"]), "image neighbour counts"
            assert np.array_equal(sol.get("flag"), out["flag"]), "MGPU boundary flags"
            assert np.array_equal(sol.get("comm_hash"), out["comm"]), "communication hash"
            stats = sol.exchange_stats()
            assert stats["boundary"] == out["count"].tolist()
            # the Sec. V cost function: pair interactions per label
            cost = np.bincount(st.label, weights=out["nreal"] + out["nimage"], minlength=scene.K)
            assert stats["cost"] == cost.astype(np.int64).tolist(), "cost per label"
            off, lst = orc.boundary_lists(st.label, out["comm"], P.dims[0] * P.dims[1] * P.dims[2], scene.K)
            assert np.array_equal(sol.get("boundary"), lst), "boundary set order"
            for f in STATE_F:
                e = _maxnorm_err(sol.get(f), getattr(st, f))
                worst[f] = max(worst[f], e)
                assert e <= tol, (k, f, e)
    finally:
        sol.close()
    return worst


def test_radix_sort_matches_stable_argsort():
    import torch
    rng = np.random.default_rng(0)
    for n, bits in [(1, 8), (4095, 8), (4096, 12), (4097, 17), (100_003, 24), (1_000_000, 27), (70_000, 32)]:
        k = rng.integers(0, 2 ** bits, size=n, dtype=np.uint64).astype(np.uint32)
        if n > 1000:
            k[: n // 3] = np.sort(k[: n // 3])      # a pre-sorted run, as after the previous step
            k[n // 2: n // 2 + 500] = 7             # a long run of equal keys
        keys = torch.from_numpy(k.view(np.int32)).cuda()
        vals = torch.arange(n, dtype=torch.int32, device="cuda")
        gsph.radix_sort_pairs(keys, vals, bits)
        torch.cuda.synchronize()
        perm = np.argsort(k, kind="stable")
        assert np.array_equal(keys.cpu().numpy().view(np.uint32), k[perm])
        assert np.array_equal(vals.cpu().numpy(), perm.astype(np.int32))
    # only the low key_bits bits decide: keys with random higher bits, digit widths 8 and 9
    for n, bits in [(50_001, 9), (70_000, 13), (65_537, 18), (9_999, 27)]:
        k = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
        keys = torch.from_numpy(k.view(np.int32)).cuda()
        vals = torch.arange(n, dtype=torch.int32, device="cuda")
        gsph.radix_sort_pairs(keys, vals, bits)
        torch.cuda.synchronize()
        perm = np.argsort(k & np.uint32((1 << bits) - 1), kind="stable")
        assert np.array_equal(vals.cpu().numpy(), perm.astype(np.int32)), bits
        assert np.array_equal(keys.cpu().numpy().view(np.uint32), k[perm]), bits


@pytest.mark.parametrize("precision,tol", [(gsph.FP64, 1e-12), (gsph.FP32_SPLIT, 2e-5)])
def test_cube_impact_lockstep(precision, tol):
    # 16^3 cube on a wall, one label: 10 steps (the cube-impact workload at its stated size)
    _lockstep(scenes.cube_impact(), precision, 10, tol)


@pytest.mark.parametrize("precision,tol", [(gsph.FP64, 1e-12), (gsph.FP32_SPLIT, 2e-5)])
def test_labels_swaps_and_boundary_lockstep(precision, tol):
    # random labels, swap heuristic every step, ragged size (not a multiple of any block size)
    s = scenes.taylor_bar(dx=0.5e-3, K=4, swap_period=1)
    assert s.n % 128 != 0
    _lockstep(s, precision, 4, tol)


def test_two_materials_per_type_swaps_lockstep():
    s = scenes.projectile_plate(dx=1e-3, plate=(20e-3, 20e-3, 4e-3), radius=3e-3, K=8, swap_period=1)
    _lockstep(s, gsph.FP64, 3, 1e-12)


def test_sixteen_labels_gravity_lockstep():
    s = scenes.collapse_block(dx=4e-3, size=(0.12, 0.06, 0.04), K=16, swap_period=2)
    _lockstep(s, gsph.FP32_SPLIT, 4, 2e-5)


@pytest.mark.parametrize("precision,tol", [(gsph.FP64, 1e-12), (gsph.FP32_SPLIT, 2e-5)])
def test_two_pass_order_lockstep(precision, tol):
    # the interaction in the order of Sec. II steps d-f: pairs within a label while the boundary set is
    # gathered into the halo buffer on a second stream, then the boundary particles' pairs across labels
    # from the halo; every bit-exact output and the state tolerance as for one pass
    s = scenes.taylor_bar(dx=0.5e-3, K=4, swap_period=1)
    _lockstep(s, precision, 4, tol, overlap=True)
    s = scenes.collapse_block(dx=4e-3, size=(0.12, 0.06, 0.04), K=16, swap_period=2)
    _lockstep(s, precision, 3, tol, overlap=True)


def test_two_pass_order_equals_one_pass():
    # the same sums in another order: neighbour counts and pair totals identical, state within rounding
    s = scenes.taylor_bar(dx=0.5e-3, K=4, swap_period=1)
    one = gsph.Solver.from_scene(s, precision=gsph.FP64, diagnostics=True)
    two = gsph.Solver.from_scene(s, precision=gsph.FP64, diagnostics=True, overlap=True)
    try:
        for _ in range(3):
            one.step(1)
            two.step(1)
        one.sync()
        two.sync()
        for f in ("id", "label", "nreal", "nimage", "flag", "boundary"):
            assert np.array_equal(one.get(f), two.get(f)), f
        assert one.exchange_stats()["pairs_total"] == two.exchange_stats()["pairs_total"]
        assert two.exchange_stats()["boundary_total"] > 0
        for f in STATE_F:
            assert _maxnorm_err(two.get(f), one.get(f)) <= 1e-13, f
    finally:
        one.close()
        two.close()


@pytest.mark.parametrize("precision,tol", [(gsph.FP64, 1e-12), (gsph.FP32_SPLIT, 2e-5)])
def test_hypervelocity_mie_gruneisen_lockstep(precision, tol):
    # Sec. IV's example at a coarse spacing: aluminium bead at 4.05 km/s, 32 degrees, onto a 2 mm plate;
    # Mie-Gruneisen EOS (compression branch at the contact) and spall cut-off, 4 labels, swaps
    s = scenes.hvi_bead_plate(dx=0.25e-3, swap_period=2)
    _lockstep(s, precision, 4, tol)


@pytest.mark.parametrize("precision,tol", [(gsph.FP64, 1e-12), (gsph.FP32_SPLIT, 2e-5)])
def test_tension_beyond_the_spall_cut_off_lockstep(precision, tol):
    # an expanding block (v = 2e6/s * x) goes into tension at once; with the cut-off at -0.3 GPa the
    # pressure of most particles is floored within the first steps (expansion branch of Mie-Gruneisen)
    s = scenes.cube_impact(n_side=10, seed=13)
    s.eos, s.p_min = [(scenes.AL6061_C0, scenes.AL6061_S, scenes.AL6061_GAMMA0)], [-3.0e8]
    c = s.pos.mean(axis=0)
    s.vel = 2.0e6 * (s.pos - c) * s.dx / s.dx
    s.walls = []
    P = orc.params_of(s)
    _lockstep(s, precision, 4, tol)
    sol = gsph.Solver.from_scene(s, precision=precision)
    try:
        sol.step(3)
        st = sol.state()
        rho = st["m"] / st["w"]
        cut = 0
        for i in range(len(rho)):
            e = st["E"][i] - 0.5 * (st["vx"][i] ** 2 + st["vy"][i] ** 2 + st["vz"][i] ** 2)
            p, _ = orc.eos(P, 0, rho[i], e)
            cut += p == -3.0e8
        assert cut > len(rho) // 2          # the floor is active for most particles
    finally:
        sol.close()


def test_adjoint_refuses_other_equations_of_state():
    s = scenes.hvi_bead_plate(dx=0.5e-3)
    sol = gsph.Solver.from_scene(s, precision=gsph.FP64, diagnostics=True)
    try:
        import torch
        lam = torch.zeros((15, s.n), dtype=torch.float64, device="cuda")
        with pytest.raises(gsph.GsphError) as ei:
            sol.adjoint_step(lam, torch.empty_like(lam), 1e-9)
        assert ei.value.code == gsph.INVALID_ARG
    finally:
        sol.close()


@pytest.mark.parametrize("precision,tol", [(gsph.FP64, 1e-12), (gsph.FP32_SPLIT, 2e-5)])
def test_heun_integrator_lockstep(precision, tol):
    # the two-stage Heun step (y* = E(y_n), y_{n+1} = (y_n + E(y*)) / 2, step-start neighbour sets):
    # wall images in both stages (cube impact), labels and swaps (Taylor bar), list overflow (dense)
    s = scenes.cube_impact(n_side=12, seed=17)
    s.integrator = 1
    _lockstep(s, precision, 4, tol)
    s = scenes.taylor_bar(dx=0.5e-3, K=4, swap_period=1)
    s.integrator = 1
    _lockstep(s, precision, 3, tol)
    s = scenes.cube_impact(n_side=10, seed=9)
    s.h = 1.6 * s.dx
    lo = tuple(v - 4 * s.h for v in s.pos.min(axis=0))
    s.grid_lo = lo
    s.grid_dims = tuple(int(np.ceil((s.pos[:, a].max() + 4 * s.h - lo[a]) / (2 * s.h))) for a in range(3))
    s.integrator = 1
    _lockstep(s, precision, 2, tol)


def _free_run_100(s):
    P = orc.params_of(s)
    st = orc.OracleState.from_scene(s)
    for _ in range(100):
        orc.step(P, st)
    sol = gsph.Solver.from_scene(s, precision=gsph.FP32_SPLIT)
    try:
        sol.step(100)
        sol.sync()
        g = sol.state()
        order = np.argsort(g["id"])
        ref = np.argsort(st.id)
        for f in STATE_F:
            e = _maxnorm_err(g[f][order], getattr(st, f)[ref])
            assert e <= 1e-3, (f, e)
    finally:
        sol.close()


def test_split_free_running_100_steps_variants():
    # the 1e-3 bound after 100 free steps for the MUSCL, Heun and varying-size variants
    s = scenes.cube_impact(n_side=12, steps=100)
    s.reconstruction = 1
    _free_run_100(s)
    s = scenes.cube_impact(n_side=12, steps=100)
    s.integrator = 1
    _free_run_100(s)
    _free_run_100(scenes.graded_block(n_side=10, nz_fine=8, nz_coarse=4, seed=6))


def test_split_free_running_100_steps():
    s = scenes.cube_impact(n_side=12, steps=100)
    P = orc.params_of(s)
    st = orc.OracleState.from_scene(s)
    for _ in range(100):
        orc.step(P, st)
    sol = gsph.Solver.from_scene(s, precision=gsph.FP32_SPLIT)
    try:
        sol.step(100)
        sol.sync()
        g = sol.state()
        order = np.argsort(g["id"])
        ref = np.argsort(st.id)
        for f in STATE_F:
            e = _maxnorm_err(g[f][order], getattr(st, f)[ref])
            assert e <= 1e-3, (f, e)
    finally:
        sol.close()


def test_conservation_on_device():
    s = scenes.cube_impact(n_side=12)
    sol = gsph.Solver.from_scene(s, precision=gsph.FP32_SPLIT)
    try:
        c0 = sol.conserved()
        sol.step(20)
        c1 = sol.conserved()
        assert abs(c1[0] - c0[0]) <= 1e-9 * c0[0]          # mass
        scale = abs(c0[3])
        assert abs(c1[1] - c0[1]) <= 1e-6 * scale and abs(c1[2] - c0[2]) <= 1e-6 * scale   # x, y momentum
        assert c1[3] > c0[3]                               # the wall pushes back
    finally:
        sol.close()


def test_particles_outside_the_grid_are_garbage():
    s = scenes.cube_impact(n_side=6)
    s.pos[:5, 2] += 1.0          # far above the grid
    sol = gsph.Solver.from_scene(s, precision=gsph.FP64, diagnostics=True)
    try:
        sol.step(1)
        st = sol.exchange_stats()
        assert st["garbage"] == 5
        key = sol.get("hash")
        C = s.grid_dims[0] * s.grid_dims[1] * s.grid_dims[2]
        assert (key[-5:] == C).all() and (key[:-5] < C).all()
        assert (sol.get("nreal")[-5:] == 0).all()
    finally:
        sol.close()


def test_hash_on_and_near_bucket_faces():
    """Positions on bucket faces, a few ulps and a few FP32 roundings either side of them, the grid's
    outer faces, far outside, NaN and infinities: the device hash (FP32 quotient with an FP64
    fallback near faces) equals the oracle's FP64 definition bit for bit, and so does the order."""
    s = scenes.cube_impact(n_side=8)
    n = s.n
    P = orc.params_of(s)
    cell, lo, dims = 2.0 * s.h, np.asarray(s.grid_lo), np.asarray(s.grid_dims)
    rng = np.random.default_rng(7)
    offs = np.array([0.0, 1e-300, 2.0 ** -60, 2.0 ** -40, 2.0 ** -30, 2.0 ** -24, 2.0 ** -22, 2.0 ** -20, 1e-4, 0.5])
    pos = np.empty((n, 3))
    for a in range(3):
        k = rng.integers(-1, dims[a] + 2, n).astype(np.float64)
        base = lo[a] + k * cell
        d = rng.choice(np.concatenate([offs, -offs]), n) * cell
        ulps = rng.integers(-3, 4, n)
        pos[:, a] = np.array([np.nextafter(b, np.inf if u > 0 else -np.inf) if u else b
                              for b, u in zip(base + d, ulps)])
        for u in range(1, 3):       # a second and third ulp step where drawn
            m = np.abs(ulps) > u
            pos[m, a] = np.nextafter(pos[m, a], np.where(ulps[m] > 0, np.inf, -np.inf))
    pos[0] = [np.nan, 0.0, 0.0]
    pos[1, 1] = np.inf
    pos[2, 2] = -np.inf
    pos[3] = lo + dims * cell          # the far corner: outside (half-open buckets)
    pos[4] = lo                        # the near corner: bucket 0
    pos[5, 0] = 1e300
    s.pos = pos
    s.vel = np.zeros_like(pos)         # one step moves nothing, only the hash is compared
    key_o = orc.hash_keys(P, pos[:, 0], pos[:, 1], pos[:, 2])
    order = orc.sort_order(key_o)
    sol = gsph.Solver.from_scene(s, precision=gsph.FP64, diagnostics=True)
    try:
        sol.step(1)
        sol.sync()
        assert np.array_equal(sol.get("hash"), key_o[order])
        assert np.array_equal(sol.get("id"), order.astype(np.uint32))
    finally:
        sol.close()


def test_invalid_label_reported():
    s = scenes.cube_impact(n_side=4)
    s.label[3] = 5               # K = 1
    c = gsph.config_from_scene(s, precision=gsph.FP64)
    sol = gsph.Solver(c)
    try:
        with pytest.raises(gsph.GsphError) as ei:
            sol.set_particles(s.pos, s.vel, s.vol, s.material, s.label)
        assert ei.value.code == gsph.DEVICE_ERROR
    finally:
        sol.close()


def test_single_particle_and_one_bucket():
    s = scenes.cube_impact(n_side=1)
    P = orc.params_of(s)
    sol = gsph.Solver.from_scene(s, precision=gsph.FP64, diagnostics=True)
    try:
        st = orc.OracleState.from_arrays(sol.state())
        orc.step(P, st)
        sol.step(1)
        for f in STATE_F:
            assert _maxnorm_err(sol.get(f), getattr(st, f)) <= 1e-12
    finally:
        sol.close()
    # many particles in a single bucket: everyone neighbours everyone
    s = scenes.cube_impact(n_side=2, jitter=0.0, dx=0.4e-3)
    s.h = 1.0e-3
    s.walls = []
    P = orc.params_of(s)
    sol = gsph.Solver.from_scene(s, precision=gsph.FP32_SPLIT, diagnostics=True)
    try:
        st = orc.OracleState.from_arrays(sol.state())
        out = orc.step(P, st)
        sol.step(1)
        assert np.array_equal(sol.get("nreal"), out["nreal"])
        assert (out["nreal"] == 7).all()
    finally:
        sol.close()


def test_empty_context_then_particle_sets_of_other_sizes():
    # a context without particles refuses the calls that need them, and an empty set is invalid
    s = scenes.taylor_bar(dx=0.8e-3, K=4, seed=5)
    P = orc.params_of(s)
    sol = gsph.Solver(gsph.config_from_scene(s, gsph.FP32_SPLIT, diagnostics=True))
    try:
        assert sol.sizes()[0] == 0
        sol.sync()
        for call in (lambda: sol.step(1), lambda: sol.swap_now(), lambda: sol.conserved(),
                     lambda: sol.dt(), lambda: sol.exchange_stats(), lambda: sol.get("x")):
            with pytest.raises(gsph.GsphError) as ei:
                call()
            assert ei.value.code == gsph.NOT_READY
        z3, z1 = np.zeros((0, 3)), np.zeros(0)
        with pytest.raises(gsph.GsphError) as ei:
            sol.set_particles(z3, z3, z1, z1.astype(np.uint8), z1.astype(np.uint8))
        assert ei.value.code == gsph.INVALID_ARG
        # the same context then takes sets of other sizes (ragged against the blocks and warps, down to
        # one particle), each stepped in lockstep with the oracle, swaps included
        n_all = s.vol.shape[0]
        for n in (n_all, 1001, 33, 1, n_all // 2 + 7):
            sol.set_particles(s.pos[:n], s.vel[:n], s.vol[:n], s.material[:n], s.label[:n])
            assert sol.sizes()[0] == n
            for k in range(2):
                st = orc.OracleState.from_arrays(sol.state())
                out = orc.step(P, st, do_swap=True, want_rates=True)
                sol.step(1)
                sol.sync()
                assert np.array_equal(sol.get("hash"), out["key"]), (n, k)
                assert np.array_equal(sol.get("id"), st.id), (n, k)
                assert np.array_equal(sol.get("label"), st.label), (n, k)
                assert np.array_equal(sol.get("nreal"), out["nreal"]), (n, k)
                assert np.array_equal(sol.get("flag"), out["flag"]), (n, k)
                for f in STATE_F:
                    e = _maxnorm_err(sol.get(f), getattr(st, f))
                    assert e <= 2e-5, (n, k, f, e)
    finally:
        sol.close()


def test_swap_now_matches_oracle_pass():
    for K, seed in ((2, 1), (5, 2), (16, 3)):
        s = scenes.taylor_bar(dx=0.4e-3, K=K, seed=seed)
        P = orc.params_of(s)
        sol = gsph.Solver.from_scene(s, precision=gsph.FP64)
        try:
            st = orc.OracleState.from_arrays(sol.state())
            moved, _ = orc.swap_pass(P, st)
            sol.swap_now()
            sol.sync()
            assert np.array_equal(sol.get("label"), st.label), K
            assert sol.exchange_stats()["swapped_last_pass"] == moved
        finally:
            sol.close()


@pytest.mark.parametrize("precision,tol", [(gsph.FP64, 1e-12), (gsph.FP32_SPLIT, 2e-5)])
def test_candidates_on_the_support_surface(precision, tol):
    # h = dx on a lattice jittered by 1e-8 dx: every interior particle has six candidates at 2 dx = 2h
    # within about 1e-8 of the support radius, far inside the FP32 rounding band, so the FP64
    # positions decide them; neighbour counts must still match the oracle bit for bit
    s = scenes.cube_impact(n_side=9, seed=11, jitter=1e-8)
    s.h = s.dx
    lo = tuple(v - 4 * s.h for v in s.pos.min(axis=0))
    s.grid_lo = lo
    s.grid_dims = tuple(int(np.ceil((s.pos[:, a].max() + 4 * s.h - lo[a]) / (2 * s.h))) for a in range(3))
    d = s.pos[:, None, :] - s.pos[None, :, :]
    rel = (d ** 2).sum(axis=2) / (2 * s.h) ** 2 - 1.0
    assert (np.abs(rel) < 3e-5).sum() > 6 * 7 ** 3        # the band is populated (ordered pairs)
    worst = _lockstep(s, precision, 3, tol)
    assert max(worst.values()) <= tol


@pytest.mark.parametrize("precision,tol", [(gsph.FP64, 1e-12), (gsph.FP32_SPLIT, 2e-5)])
def test_dense_neighbourhoods_beyond_list_capacity(precision, tol):
    # h = 1.6 dx: about 137 neighbours per interior particle, more than the per-particle list holds,
    # so the remainder goes through the re-scan path; counts and state must still match
    s = scenes.cube_impact(n_side=10, seed=9)
    s.h = 1.6 * s.dx
    lo = tuple(v - 4 * s.h for v in s.pos.min(axis=0))
    s.grid_lo = lo
    s.grid_dims = tuple(int(np.ceil((s.pos[:, a].max() + 4 * s.h - lo[a]) / (2 * s.h))) for a in range(3))
    worst = _lockstep(s, precision, 2, tol)
    assert max(worst.values()) <= tol
