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
    rec = adjoint.ForwardRecord(s, steps=20, every=5, precision=gsph.FP64)
    g = rec.gradient()
    rec.close()
    P = orc.params_of(s)
    st = orc.OracleState.from_scene(s)
    J, go = orc.forward_gradient(P, st, rec.dts, adjoint.rear_face_ids(s))
    assert rec.J == pytest.approx(J, rel=1e-10)
    for k in range(3):
        assert g[k] == pytest.approx(go[k], rel=1e-6, abs=1e-12 * abs(go).max()), (k, g, go)


def _J_fp64(scene, dts):
    sol = gsph.Solver.from_scene(scene, precision=gsph.FP64)
    for dt in dts:
        sol.set_dt(dt)
        sol.step(1)
    sol.sync()
    ids = sol.get("id")
    vz = sol.get("vz")
    J = float(vz[np.isin(ids, adjoint.rear_face_ids(scene))].mean())
    sol.close()
    return J


def test_adjoint_workload_gradient_against_finite_differences():
    base = scenes.adjoint_cube()          # 64^3 = 262,144 particles
    Y0, G0, v00 = base.materials[0][3], base.materials[0][2], float(base.vel[0, 2])
    rec = adjoint.ForwardRecord(base, steps=200, every=20, precision=gsph.FP32_SPLIT)
    g = rec.gradient()
    dts = rec.dts
    rec.close()
    for k, (name, val) in enumerate((("Y", Y0), ("G", G0), ("v0", v00))):
        e = 1e-4 * abs(val)
        args = lambda d: dict(Y=Y0 + (d if k == 0 else 0.0), G=G0 + (d if k == 1 else 0.0),
                              v0=v00 + (d if k == 2 else 0.0))
        Jp = _J_fp64(adjoint.with_parameters(base, **args(e)), dts)
        Jm = _J_fp64(adjoint.with_parameters(base, **args(-e)), dts)
        fd = (Jp - Jm) / (2 * e)
        assert g[k] == pytest.approx(fd, rel=1e-4), (name, g[k], fd)


def test_autograd_function_backward():
    import torch
    base = scenes.cube_impact(n_side=6, seed=3)
    theta = torch.tensor([150.0e6, base.materials[0][2], -120.0], dtype=torch.float64, requires_grad=True)
    J = adjoint.impact_observable(base, theta, steps=12, every=4, precision=gsph.FP64)
    J.backward()
    rec = adjoint.ForwardRecord(adjoint.with_parameters(base, 150.0e6, base.materials[0][2], -120.0),
                                steps=12, every=4, precision=gsph.FP64)
    g = rec.gradient()
    rec.close()
    assert float(J) == pytest.approx(rec.J, rel=1e-14)
    assert np.allclose(theta.grad.numpy(), g, rtol=1e-12, atol=0.0)
    assert np.all(theta.grad.numpy() != 0.0)
