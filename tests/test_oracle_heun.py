"""Pin of the second-order integrator reading (two-stage Heun in its strong-stability-preserving
form, both stages over the neighbour set of the step's start): on a smooth elastic problem whose
neighbour set does not change, halving the time step shrinks the difference between successive
refinements about 4 times (second order), against about 2 times for forward Euler."""
import numpy as np
import pytest

from oracle import orc
from paper_2310_03596_gb300 import scenes


def _run(integrator: int, nsteps: int, T: float):
    s = scenes.cube_impact(n_side=8, seed=21, speed=0.0)
    s.walls = []
    # a smooth shear-and-compression velocity field of 2 m/s (displacements far below the spacing)
    c = s.pos.mean(axis=0)
    L = np.ptp(s.pos[:, 0])
    s.vel = np.zeros_like(s.pos)
    s.vel[:, 0] = 2.0 * np.sin(np.pi * (s.pos[:, 1] - c[1]) / L)
    s.vel[:, 2] = 2.0 * np.cos(np.pi * (s.pos[:, 0] - c[0]) / L)
    s.integrator = integrator
    P = orc.params_of(s)
    st = orc.OracleState.from_scene(s)
    for _ in range(nsteps):
        orc.step(P, st, dt=T / nsteps)
    order = np.argsort(st.id)
    return np.concatenate([getattr(st, f)[order] for f in ("vx", "vz", "sxy", "sxz", "E")])


@pytest.mark.parametrize("integrator,expect", [(0, 2.0), (1, 4.0)])
def test_convergence_order(integrator, expect):
    T = 4.0e-7                  # about 6 CFL steps of the coarsest run
    y = [_run(integrator, n, T) for n in (4, 8, 16)]
    ratio = np.abs(y[0] - y[1]).max() / np.abs(y[1] - y[2]).max()
    assert ratio == pytest.approx(expect, rel=0.15), ratio


def test_heun_matches_euler_to_first_order():
    # both integrate the same rates: one step differs by O(dt^2), i.e. much less than the change
    T = 1.0e-8
    e, h, y0 = _run(0, 1, T), _run(1, 1, T), _run(0, 1, 1e-30)
    assert np.abs(h - e).max() < 0.05 * np.abs(e - y0).max()
