"""Pins of the oracle's equations of state (Sec. IV names a Mie-Gruneisen EOS with a spall cut-off;
the form is a reading) against facts that do not come from the oracle's formula:

- the Rankine-Hugoniot jump conditions of a steady shock with the linear relation Us = c0 + s up
  (mass: rho0 Us = rho (Us - up); momentum: p = rho0 Us up; energy: e = up^2 / 2 from rest): a state
  built from them lies on the reference curve, so the EOS returns that pressure whatever gamma0 is;
- the Gruneisen definition dp/de at fixed density = Gamma rho = gamma0 rho0;
- the isentropic sound speed c_b^2 = dp/drho along de = (p / rho^2) drho, by central differences;
- the rest state: p(rho0, 0) = 0 with c_b = c0;
- the cut-off floors tension at p_min and leaves the sound speed of the uncut EOS;
- the linear EOS: p = K (rho/rho0 - 1) and c_b^2 = K / rho.
"""
import math

import pytest

from oracle import orc
from paper_2310_03596_gb300 import scenes

RHO0, C0, S, G0 = scenes.AL6061_RHO0, scenes.AL6061_C0, scenes.AL6061_S, scenes.AL6061_GAMMA0


def _params(gamma0=G0, p_min=-math.inf, s=S):
    sc = scenes.hvi_bead_plate(dx=0.5e-3)
    sc.eos = [(C0, s, gamma0)]
    sc.p_min = [p_min]
    return orc.params_of(sc)


@pytest.mark.parametrize("gamma0", [0.0, 1.0, G0, 3.0])
def test_states_of_the_rankine_hugoniot_jump(gamma0):
    P = _params(gamma0)
    for up in (10.0, 200.0, 1000.0, 2500.0, 4000.0):
        us = C0 + S * up
        rho = RHO0 * us / (us - up)
        e = 0.5 * up * up
        p, _ = orc.eos(P, 0, rho, e)
        assert p == pytest.approx(RHO0 * us * up, rel=1e-12), (gamma0, up)


def test_energy_derivative_is_the_gruneisen_coefficient():
    P = _params()
    for rho in (0.9 * RHO0, RHO0, 1.2 * RHO0):
        p0, _ = orc.eos(P, 0, rho, 1.0e4)
        p1, _ = orc.eos(P, 0, rho, 3.0e5)
        assert (p1 - p0) / (3.0e5 - 1.0e4) == pytest.approx(G0 * RHO0, rel=1e-9)


@pytest.mark.parametrize("rho_over,e", [(1.0, 0.0), (1.05, 2.0e4), (1.3, 5.0e5), (0.95, 1.0e4), (0.8, 0.0)])
def test_sound_speed_is_the_isentropic_derivative(rho_over, e):
    P = _params()
    rho = rho_over * RHO0
    p, cb2 = orc.eos(P, 0, rho, e)
    d = 1e-6 * rho
    pp, _ = orc.eos(P, 0, rho + d, e + p * d / rho ** 2)
    pm, _ = orc.eos(P, 0, rho - d, e - p * d / rho ** 2)
    assert cb2 == pytest.approx((pp - pm) / (2 * d), rel=1e-6)


def test_rest_state():
    P = _params()
    p, cb2 = orc.eos(P, 0, RHO0, 0.0)
    assert p == 0.0
    assert math.sqrt(cb2) == pytest.approx(C0, rel=1e-14)


def test_cut_off_floors_tension_only():
    cut = -1.2e9
    Pc, Pn = _params(p_min=cut), _params()
    for rho, e in ((0.7 * RHO0, 0.0), (0.8 * RHO0, 1.0e4)):
        pn, cn = orc.eos(Pn, 0, rho, e)
        pc, cc = orc.eos(Pc, 0, rho, e)
        assert pn < cut and pc == cut and cc == cn
    for rho, e in ((0.99 * RHO0, 0.0), (1.2 * RHO0, 1.0e5)):
        assert orc.eos(Pc, 0, rho, e) == orc.eos(Pn, 0, rho, e)


def test_linear_equation_of_state():
    sc = scenes.cube_impact(n_side=2)
    P = orc.params_of(sc)
    rho0, K = sc.materials[0][0], sc.materials[0][1]
    for rho in (0.9 * rho0, rho0, 1.1 * rho0):
        p, cb2 = orc.eos(P, 0, rho, 123.0)
        assert p == pytest.approx(K * (rho / rho0 - 1.0), rel=1e-15, abs=1e-6)
        assert cb2 == pytest.approx(K / rho, rel=1e-15)


def test_signal_speed_tracks_the_eos():
    # the time step's sound speed against the FP64 EOS of one particle at rest, compressed and
    # heated: c = sqrt(c_b^2 + 4G / (3 rho)) to FP64 rounding
    sc = scenes.hvi_bead_plate(dx=0.5e-3)
    P = orc.params_of(sc)
    G = sc.materials[0][2]
    for rho_over, e in ((1.0, 0.0), (1.25, 4.0e5), (0.9, 1.0e4)):
        st = orc.OracleState(1)
        st.x[:] = 0.0
        st.w[:] = 1e-9
        st.m[:] = rho_over * RHO0 * 1e-9
        st.E[:] = e
        st.mat[:] = 0
        dt = orc.dt(P, st)
        _, cb2 = orc.eos(P, 0, rho_over * RHO0, e)
        c = math.sqrt(cb2 + 4 * G / (3 * rho_over * RHO0))
        assert sc.cfl * sc.h / dt == pytest.approx(c, rel=1e-14), (rho_over, e)
