"""Pin of the oracle's forward-mode gradient of the impact observable (mean z velocity of the rear
face) w.r.t. yield stress, shear modulus and initial z velocity, with the dt schedule frozen to the
unperturbed run, against central finite differences of the plain FP64 forward run (step 1e-4
relative)."""
import numpy as np
import pytest

from oracle import orc
from paper_2310_03596_gb300 import scenes

Y0, G0 = scenes.ALUMINIUM[3], scenes.ALUMINIUM[2]


def _setup(Y=Y0, G=G0, v0=-100.0, n_side=6):
    s = scenes.cube_impact(n_side=n_side, seed=3)
    rho0, K, _, _ = s.materials[0]
    s.materials = [(rho0, K, G, Y)]
    s.vel[:, 2] = v0
    return s, orc.params_of(s), orc.OracleState.from_scene(s)


def _J(dts, obs, **kw):
    s, P, st = _setup(**kw)
    for dt in dts:
        r, _, _ = orc.rates(P, st)
        orc.integrate(P, st, r, dt)
    return st.vz[np.isin(st.id, obs)].mean()


def test_forward_gradient_matches_central_differences():
    n_side, nsteps = 6, 20
    s, P, st = _setup(n_side=n_side)
    run = st.copy()
    dts = []
    for _ in range(nsteps):
        dts.append(orc.dt(P, run))
        r, _, _ = orc.rates(P, run)
        orc.integrate(P, run, r, dts[-1])
    rear = np.rint(s.pos[:, 2] / s.dx - 0.5).astype(int) == n_side - 1
    obs = np.where(rear)[0].astype(np.uint32)
    J, g = orc.forward_gradient(P, st.copy(), dts, obs)
    assert J == pytest.approx(run.vz[np.isin(run.id, obs)].mean(), rel=1e-14)
    for k, (name, base) in enumerate((("Y", Y0), ("G", G0), ("v0", -100.0))):
        e = 1e-4 * abs(base)
        kw = lambda d: {name: base + d}
        fd = (_J(dts, obs, **kw(e)) - _J(dts, obs, **kw(-e))) / (2 * e)
        assert g[k] == pytest.approx(fd, rel=1e-4), name
