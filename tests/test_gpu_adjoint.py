"""GPU adjoint (reverse mode of interaction + integration) against finite differences and against the
oracle's forward-mode gradient.

- One adjoint step is the transpose of the FP64 step's Jacobian (neighbour set and dt fixed): for
  random lam and delta, lam . (Step(y + e delta) - Step(y - e delta)) / 2e = (Step^T lam) . delta.
- dJ/d(Y, G, v0) of the rear-face mean z velocity equals the oracle's dual-number gradient.
- The adjoint workload as stated (64^3 cube, 200 steps, FP32-split forward, checkpoint every 20):
  gradient within 1e-4 of central finite differences (step 1e-4 relative) of the FP64 forward with
  the dt schedule frozen.
"""
import numpy as np
import pytest

from oracle import orc
from paper_2310_03596_gb300 import adjoint, gsph, scenes

pytestmark = pytest.mark.gpu

STATE = tuple(gsph.FIELDS[:15])


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _state_by_id(sol):
    st = sol.state()
    order = np.argsort(st["id"])
    return np.stack([st[f][order] for f in STATE]), st


def test_adjoint_step_is_the_transposed_step_jacobian():
    import torch
    s = scenes.cube_impact(n_side=8, seed=4)
    sol = gsph.Solver.from_scene(s, precision=gsph.FP64, diagnostics=True)
    sol.step(6)                      # plastic flow has started at the wall
    sol.sync()
    y0 = sol.state()
    dt = sol.dt()
    n = s.n
    rng = np.random.default_rng(0)
    # field scales of the state, so that every component is exercised at a comparable size
    scale = np.array([np.abs(y0[f]).max() + 1e-30 for f in STATE])
    scale[:3] = s.dx
    lam_id = rng.standard_normal((15, n)) / scale[:, None]     # adjoint, indexed by persistent id
    delta = rng.standard_normal((15, n)) * scale[:, None]      # perturbation, in y0's slot order
    eps = 1e-7
    outs = []
    for sgn in (1.0, -1.0):
        for k, f in enumerate(STATE):
            sol.put(f, y0[f] + sgn * eps * delta[k])
        for f in ("material", "label", "id"):
            sol.put(f, y0[f])
        sol.set_dt(dt)
        sol.step(1)
        yb, _ = _state_by_id(sol)
        outs.append(yb)
    fd = float((lam_id * (outs[0] - outs[1])).sum() / (2 * eps))
    # adjoint at y0: lam_next in the slot order of the step's output (the hash order of this step)
    for f in STATE + ("material", "label", "id"):
        sol.put(f, y0[f])
    sol.set_dt(dt)
    sol.step(1)
    ids_out = sol.get("id")
    for f in STATE + ("material", "label", "id"):
        sol.put(f, y0[f])
    lam_next = torch.from_numpy(np.ascontiguousarray(lam_id[:, ids_out])).cuda()
    lam_prev = torch.empty_like(lam_next)
    sol.adjoint_step(lam_next, lam_prev, dt)
    ad = float((lam_prev.cpu().numpy() * delta).sum())
    assert ad == pytest.approx(fd, rel=1e-6), (ad, fd)
    sol.close()


def test_gradient_matches_oracle_forward_mode():
    base = scenes.cube_impact(n_side=6, seed=3)
    Y0, G0 = 150.0e6, base.materials[0][2]
    s = adjoint.with_parameters(base, Y0, G0, -120.0)
    J, g, dts = adjoint.observable(s, steps=20, every=5, precision=gsph.FP64)
    P = orc.params_of(s)
    st = orc.OracleState.from_scene(s)
    Jo, go = orc.forward_gradient(P, st, dts, adjoint.rear_face_ids(s))
    assert J == pytest.approx(Jo, rel=1e-10)
    for k in range(3):
        assert g[k] == pytest.approx(go[k], rel=1e-6, abs=1e-12 * abs(go).max()), (k, g, go)


def test_adjoint_leaves_the_final_state_and_replays_bit_for_bit():
    # the call advances the context by `steps` steps: its state equals that of plain steps with the same
    # schedule, bit for bit (the recomputed segments and the restore do not disturb it)
    s = scenes.cube_impact(n_side=8, seed=6, K=2)
    s.swap_period = 3
    a = gsph.Solver.from_scene(s, precision=gsph.FP32_SPLIT)
    J, g, dts = a.adjoint(11, 4, adjoint.rear_face_ids(s))
    b = gsph.Solver.from_scene(s, precision=gsph.FP32_SPLIT)
    for dt in dts:
        b.set_dt(dt)
        b.step(1)
    b.sync()
    sa, sb = a.state(), b.state()
    for f in STATE + ("id", "label"):
        assert np.array_equal(sa[f], sb[f]), f
    a.close()
    b.close()


def test_adjoint_workload_gradient_against_finite_differences():
    base = scenes.adjoint_cube()          # 64^3 = 262,144 particles
    Y0, G0, v00 = base.materials[0][3], base.materials[0][2], float(base.vel[0, 2])
    J0, g, dts = adjoint.observable(base, steps=200, every=20, precision=gsph.FP32_SPLIT)
    live = []
    for k, (name, val) in enumerate((("Y", Y0), ("G", G0), ("v0", v00))):
        e = 1e-4 * abs(val)
        args = lambda d: dict(Y=Y0 + (d if k == 0 else 0.0), G=G0 + (d if k == 1 else 0.0),
                              v0=v00 + (d if k == 2 else 0.0))
        # J on the frozen schedule (its definition), forward in FP64
        Jp, _, _ = adjoint.observable(adjoint.with_parameters(base, **args(e)), 200, 20, gsph.FP64, dts=dts,
                                      want_gradient=False)
        Jm, _, _ = adjoint.observable(adjoint.with_parameters(base, **args(-e)), 200, 20, gsph.FP64, dts=dts,
                                      want_gradient=False)
        fd = (Jp - Jm) / (2 * e)
        assert g[k] == pytest.approx(fd, rel=1e-4), (name, g[k], fd)
        # for the record: the same difference with each run's own CFL steps (the time step's own
        # dependence on G and v0, which the frozen schedule leaves out)
        Lp, _, _ = adjoint.observable(adjoint.with_parameters(base, **args(e)), 200, 20, gsph.FP64,
                                      want_gradient=False)
        Lm, _, _ = adjoint.observable(adjoint.with_parameters(base, **args(-e)), 200, 20, gsph.FP64,
                                      want_gradient=False)
        live.append((name, g[k], (Lp - Lm) / (2 * e)))
    print("frozen-schedule gradient vs central difference with live CFL steps:",
          [(nm, gk, fl, abs(gk - fl) / max(abs(fl), 1e-300)) for nm, gk, fl in live])
    for nm, gk, fl in live:
        assert np.isfinite(fl)


def test_autograd_function_backward():
    import torch
    base = scenes.cube_impact(n_side=6, seed=3)
    theta = torch.tensor([150.0e6, base.materials[0][2], -120.0], dtype=torch.float64, requires_grad=True)
    J = adjoint.impact_observable(base, theta, steps=12, every=4, precision=gsph.FP64)
    J.backward()
    J2, g, _ = adjoint.observable(adjoint.with_parameters(base, 150.0e6, base.materials[0][2], -120.0),
                                  steps=12, every=4, precision=gsph.FP64)
    assert J.item() == pytest.approx(J2, rel=1e-14)
    assert np.allclose(theta.grad.numpy(), g, rtol=1e-12, atol=0.0)
    assert np.all(theta.grad.numpy() != 0.0)


def test_state_blob_round_trip_resumes_bit_for_bit():
    import torch
    # checkpoint / resume: a blob saved after 5 steps, loaded into a fresh context, continues exactly
    # like the original (host and device blobs; a blob of another size reallocates the context)
    s = scenes.cube_impact(n_side=10, seed=9, K=3)
    s.swap_period = 2
    a = gsph.Solver.from_scene(s, precision=gsph.FP32_SPLIT)
    a.step(5)
    host = a.save_state()
    dev = a.save_state(torch.empty(a.state_bytes(), dtype=torch.uint8, device="cuda"))
    a.step(6)
    a.sync()
    want = a.state()
    # the same configuration with a smaller particle set (the blob carries the state, not the config)
    import copy
    other = copy.deepcopy(s)
    for f in ("pos", "vel", "vol", "material", "label"):
        setattr(other, f, getattr(s, f)[:100].copy())
    for blob in (host, dev):
        b = gsph.Solver.from_scene(other, precision=gsph.FP32_SPLIT)
        b.load_state(blob)
        assert b.n == s.n
        b.step(6)
        b.sync()
        got = b.state()
        for f in STATE + ("id", "label", "material"):
            assert np.array_equal(got[f], want[f]), f
        b.close()
    bad = host.copy()
    bad[0] ^= 1
    with pytest.raises(gsph.GsphError):
        a.load_state(bad)
    a.close()
