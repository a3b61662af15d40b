"""The GPU side of the label-sharded data plane on one GPU: the exchange bookkeeping (bucket hash, label
masks, MGPU flags, fixed-point Cg coordinates, balancing hashes) on CUDA tensors equals the CPU tensors'
and the oracle's bit for bit, and the libgsph interaction engine advances a rank's own particles against
own + halo particles as the oracle does (FP64 within 1e-12; dt and neighbour counts exact). (The
multi-rank exchanges themselves are covered by the gloo tests on CPU: ranks that wait on each other do
not run on one GPU.)"""
import numpy as np
import pytest
import torch

from oracle import orc
from paper_2310_03596_gb300 import gsph, scenes, sharded

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _tensors(st, dev):
    d = {f: torch.as_tensor(np.ascontiguousarray(getattr(st, f)), device=dev) for f in orc.FIELDS}
    d["mat"] = torch.as_tensor(st.mat, device=dev)
    d["label"] = torch.as_tensor(st.label, device=dev)
    d["id"] = torch.as_tensor(st.id.astype(np.int64), device=dev)
    return d


def test_bookkeeping_on_cuda_equals_cpu_and_oracle():
    s = scenes.cube_impact(n_side=12, K=3, seed=21)
    G = sharded.Grid(s)
    P = orc.params_of(s)
    st = orc.OracleState.from_scene(s)
    st.x += 0.3e-3 * np.sin(st.y * 1e3)     # off the lattice
    res = {}
    for dev in ("cpu", "cuda"):
        t = _tensors(st, dev)
        key = sharded.bucket_keys(G, t["x"], t["y"], t["z"])
        mask = sharded.label_mask(G, key, t["label"].to(torch.int64))
        flag = sharded.boundary_flags(G, key, t["label"].to(torch.int64), mask)
        q = [sharded.fixed_point(G, t[c], a) for a, c in enumerate(("x", "y", "z"))]
        M, d = [0.006, 0.005, 0.004], [0.002, -0.001, 0.0005]
        dn = float(np.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]))
        hb = sharded.balancing_hash(M, d, dn, dn * 0.5, t["x"], t["y"], t["z"])
        res[dev] = [v.cpu().numpy() for v in (key, mask, flag, *q, hb)]
    for a, b in zip(res["cpu"], res["cuda"]):
        assert np.array_equal(a, b)
    key, _, flag = res["cpu"][:3]
    assert np.array_equal(key, orc.hash_keys(P, st.x, st.y, st.z).astype(np.int64))
    oflag, _, _ = orc.comm_hash(P, orc.hash_keys(P, st.x, st.y, st.z), st.label)
    assert np.array_equal(flag.astype(np.uint8), oflag)
    own = np.array([0.006, 0.005, 0.004]) - 0.5 * np.array([0.002, -0.001, 0.0005])
    oth = own + np.array([0.002, -0.001, 0.0005])
    hb = res["cpu"][-1]
    for i in range(0, st.n, 97):
        assert hb[i] == orc.balancing_hash(own, oth, [st.x[i], st.y[i], st.z[i]]), i


def test_gpu_engine_advances_own_particles_like_the_oracle():
    s = scenes.cube_impact(n_side=10, K=2, seed=4)
    P = orc.params_of(s)
    st = orc.OracleState.from_scene(s)
    sol = gsph.Solver.from_scene(s, precision=gsph.FP64)
    sol.step(3)                                 # a state with stress and plastic flow at the wall
    sol.sync()
    st = orc.OracleState.from_arrays(sol.state())
    sol.close()
    G = sharded.Grid(s)
    t = _tensors(st, "cuda")
    key = sharded.bucket_keys(G, t["x"], t["y"], t["z"])
    lab = t["label"].to(torch.int64)
    mask = sharded.label_mask(G, key, lab)
    flag = sharded.boundary_flags(G, key, lab, mask)
    own = lab == 0
    union = sharded._cat([sharded._take(t, own), sharded._take(t, (~own) & flag)])
    n_own = int(own.sum())
    dt = orc.dt(P, st)
    eng = sharded.GpuEngine(s, gsph.FP64)
    new, nr, ni = eng.advance(union, n_own, dt)
    # the oracle: rates of the own particles over the whole set, then their integration
    r, onr, oni = orc.rates(P, st)
    sel = np.where(st.label == 0)[0]
    ost = orc.OracleState.from_arrays({f: v[sel] for f, v in st.arrays().items()})
    orc.integrate(P, ost, r[sel], dt)
    o = np.argsort(new["id"].cpu().numpy())
    oo = np.argsort(ost.id)
    assert np.array_equal(new["id"].cpu().numpy()[o], ost.id[oo].astype(np.int64))
    assert np.array_equal(nr.cpu().numpy()[o], onr[sel][oo])
    assert np.array_equal(ni.cpu().numpy()[o], oni[sel][oo])
    for f in orc.FIELDS:
        want = getattr(ost, f)[oo]
        got = new[f].cpu().numpy()[o]
        assert np.abs(got - want).max() <= 1e-12 * max(np.abs(want).max(), 1e-300), f
    own_t = sharded._take(t, own)
    assert eng.dt(own_t) == orc.dt(P, orc.OracleState.from_arrays({f: v[sel] for f, v in st.arrays().items()}))
