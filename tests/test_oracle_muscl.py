"""Pins of the MUSCL reconstruction reading (the second-order SPH-ALE variant; the paper gives no
scheme): gradients of v and sigma = -p I + S by the SPH gradient operator over real and image
neighbours, minmod-limited linear reconstruction of v and sigma at the pair midpoint, density, energy
and impedance at the particle values, transport velocity = particle velocity.

- the gradient of a linear field on a perfect lattice is A M with M the lattice moment
  sum_k w (k dx) (x) grad W, summed here over the lattice offsets independently of the oracle;
- uniform fields have zero gradients, and then the reconstructed scheme gives the first-order rates;
- a body on a mirror wall gives the same gradients and rates as the same body doubled by its mirror
  image with no wall (the image states and image gradients);
- the reconstructed fluxes stay antisymmetric: mass, momentum and energy are conserved on a free body;
- on a linear velocity field with zero stress the first-order Riemann states heat the interior (the
  acoustic dissipation of the jump u_R - u_L); the reconstructed jump, and with it the heating, is
  (1 - m) times smaller, m the lattice moment of the SPH gradient (0.979 at h = 1.3 dx).
"""
import numpy as np

from oracle import orc
from paper_2310_03596_gb300 import scenes


def _state(n_side=9, jitter=0.0, walls=(), seed=0, dx=1e-3, muscl=1):
    s = scenes.cube_impact(n_side=n_side, jitter=jitter, seed=seed, dx=dx)
    s.walls = list(walls)
    s.reconstruction = muscl
    return s, orc.params_of(s), orc.OracleState.from_scene(s)


def _interior(s, margin=3):
    idx = np.rint(s.pos / s.dx - 0.5).astype(int)
    n = round(s.n ** (1 / 3))
    return ((idx >= margin) & (idx <= n - 1 - margin)).all(axis=1)


def _lattice_moment(h, dx):
    # M_eb = sum over lattice offsets k != 0 within 2h of w (x_j - x_i)_e (grad_i W_ij)_b with
    # grad_i W_ij = |dW/dr| (x_j - x_i) / r
    m = int(np.ceil(2 * h / dx))
    M = np.zeros((3, 3))
    for i in range(-m, m + 1):
        for j in range(-m, m + 1):
            for k in range(-m, m + 1):
                d = dx * np.array([i, j, k], float)
                r = np.sqrt(d @ d)
                if r == 0 or not r < 2 * h:
                    continue
                M += dx ** 3 * np.outer(d, orc.kernel_dw(r, h) * d / r)
    return M


def test_gradient_of_linear_fields_is_the_lattice_moment():
    s, P, st = _state(n_side=11)
    X = np.stack([st.x, st.y, st.z], 1)
    A = np.array([[10.0, -40.0, 5.0], [0.0, 20.0, 30.0], [-15.0, 7.0, -30.0]])
    V = X @ A.T
    st.vx[:], st.vy[:], st.vz[:] = V[:, 0], V[:, 1], V[:, 2]
    B = np.array([[1e9, 2e9, -3e9], [-2e9, 0.5e9, 1e9], [0.0, 0.0, 0.0],
                  [3e9, -1e9, 2e9], [0.0, 1e9, 0.0], [-1e9, -1e9, 4e9]])
    B[2] = -(B[0] + B[1])                              # S traceless everywhere
    for q, f in enumerate(("sxx", "syy", "szz", "sxy", "sxz", "syz")):
        getattr(st, f)[:] = X @ B[q]
    G = orc.gradients(P, st)
    M = _lattice_moment(s.h, s.dx)
    assert np.abs(M - np.eye(3)).max() < 0.05          # the SPH gradient is nearly exact on the lattice
    inn = _interior(s)
    assert inn.sum() > 0
    exp_v = A @ M
    got_v = G[inn, :9].reshape(-1, 3, 3)
    assert np.abs(got_v - exp_v).max() <= 1e-10 * np.abs(exp_v).max()
    # uniform density: p is uniform, so grad sigma = grad S
    exp_s = B @ M
    got_s = G[inn, 9:].reshape(-1, 6, 3)
    assert np.abs(got_s - exp_s).max() <= 1e-10 * np.abs(exp_s).max()


def test_uniform_fields_have_zero_gradients_and_first_order_rates():
    s, P, st = _state(n_side=8, jitter=0.01, walls=[(2, 0.0)])
    st.vx[:] = 12.0; st.vy[:] = -7.0; st.vz[:] = -30.0
    st.sxx[:] = 3e7; st.syy[:] = -1e7; st.szz[:] = -2e7; st.sxy[:] = 5e6; st.sxz[:] = -4e6; st.syz[:] = 1e6
    st.E[:] = 1e5
    G = orc.gradients(P, st)
    inner = np.abs(G[:, :9]).max(axis=1)
    # away from the wall every difference phi_j - phi_i is exactly zero
    far = st.z > 3 * s.h
    assert far.sum() > 0 and (G[far] == 0.0).all()
    r1, _, _ = orc.rates(P, st)
    s.reconstruction = 0
    r0, _, _ = orc.rates(orc.params_of(s), st)
    # the wall images mirror v_z and the shear stresses, so near the wall the gradients are nonzero;
    # the reconstructed and first-order rates then differ there only
    scale = np.abs(r0).max(axis=0)
    for k in range(orc.NRATE):
        if scale[k] > 0:
            assert np.abs(r1[far, k] - r0[far, k]).max() <= 1e-12 * scale[k], k
    assert inner[~far].max() > 0


def _doubled(s, st):
    """The body and its mirror image in the plane z = 0, with the mirrored state and no wall."""
    d = {k: v.copy() for k, v in st.arrays().items()}
    m = {k: v.copy() for k, v in st.arrays().items()}
    m["z"] = -m["z"]
    m["vz"] = -m["vz"]
    m["sxz"] = -m["sxz"]
    m["syz"] = -m["syz"]
    m["id"] = m["id"] + st.n
    both = {k: np.concatenate([d[k], m[k]]) for k in d}
    s2 = scenes.cube_impact(n_side=round(st.n ** (1 / 3)), jitter=0.0, dx=s.dx)
    s2.walls = []
    s2.reconstruction = s.reconstruction
    lo = list(s2.grid_lo)
    top = lo[2] + s2.grid_dims[2] * 2 * s2.h
    nz = int(np.ceil((top + (top - 0.0)) / (2 * s2.h)))
    lo[2] = top - nz * 2 * s2.h
    s2.grid_lo = tuple(lo)
    dims = list(s2.grid_dims)
    dims[2] = nz
    s2.grid_dims = tuple(dims)
    return orc.params_of(s2), orc.OracleState.from_arrays(both)


def test_mirror_wall_equals_doubled_body():
    s, P, st = _state(n_side=7, jitter=0.01, walls=[(2, 0.0)])
    rng = np.random.default_rng(5)
    X = np.stack([st.x, st.y, st.z], 1)
    # smooth, non-symmetric fields: the images carry nonzero gradients of every kind
    st.vx[:] = 20.0 * np.sin(900.0 * X[:, 2]) + 3.0
    st.vy[:] = 10.0 * np.cos(700.0 * X[:, 0])
    st.vz[:] = -40.0 + 15.0 * np.sin(800.0 * X[:, 1] + 500.0 * X[:, 2])
    for f, a in (("sxx", 2e7), ("syy", -1e7), ("sxy", 3e7), ("sxz", -2e7), ("syz", 1e7)):
        getattr(st, f)[:] = a * np.cos(600.0 * X[:, 2] + rng.random())
    st.szz[:] = -(st.sxx + st.syy)
    st.m[:] = st.m * (1.0 + 0.01 * np.sin(1000.0 * X[:, 2]))
    P2, st2 = _doubled(s, st)
    G = orc.gradients(P, st)
    G2 = orc.gradients(P2, st2)[: st.n]
    assert np.abs(G - G2).max() <= 1e-9 * np.abs(G).max()
    r, _, ni = orc.rates(P, st)
    r2, _, _ = orc.rates(P2, st2)
    assert ni.sum() > 0
    scale = np.abs(r).max(axis=0)
    for k in range(orc.NRATE):
        assert np.abs(r[:, k] - r2[: st.n, k]).max() <= 1e-9 * scale[k], k


def test_reconstructed_fluxes_conserve_on_a_free_body():
    s, P, st = _state(n_side=9, jitter=0.01)
    rng = np.random.default_rng(3)
    X = np.stack([st.x, st.y, st.z], 1)
    st.vx[:] = 20.0 * np.sin(800.0 * X[:, 1]) + rng.normal(0, 2.0, st.n)
    st.vy[:] = 10.0 * np.cos(600.0 * X[:, 2]) + rng.normal(0, 2.0, st.n)
    st.vz[:] = 30.0 * np.sin(700.0 * X[:, 0]) + rng.normal(0, 2.0, st.n)
    for f in ("sxx", "syy", "sxy", "sxz", "syz"):
        getattr(st, f)[:] = rng.normal(0, 3e7, st.n)
    st.szz[:] = -(st.sxx + st.syy)
    st.E[:] = 1e4 * rng.random(st.n) + 0.5 * (st.vx ** 2 + st.vy ** 2 + st.vz ** 2)
    r, _, _ = orc.rates(P, st)
    for k in (1, 2, 3, 4, 5):
        assert abs(r[:, k].sum()) <= 1e-13 * np.abs(r[:, k]).sum(), k


def _heating(s, st, muscl):
    s.reconstruction = muscl
    r, _, _ = orc.rates(orc.params_of(s), st)
    v = np.stack([st.vx, st.vy, st.vz], 1)
    dm, dmv, dmE = r[:, 1], r[:, 2:5], r[:, 5]
    # m de/dt = (d(mE) - E dm) - v . (d(mv) - v dm)
    return (dmE - st.E * dm) - np.einsum("ij,ij->i", v, dmv - v * dm[:, None])


def test_reconstruction_scales_the_acoustic_dissipation_by_the_gradient_error():
    # sigma = 0 and equal impedances: the only interface traction is t* = Z (u_R - u_L) / 2, and the
    # heating is the work of t* on the pair's relative motion. For v = A x on the perfect lattice every
    # interior pair's slope is G . d = m (A d) with m = M_xx < 1 (M = m I): minmod keeps the slope,
    # the reconstructed jump is (1 - m) times the particle jump, and so is the heating, exactly.
    # (Interior: two supports from the surface, so that the neighbours' gradients are complete too.)
    s, P, st = _state(n_side=11)
    X = np.stack([st.x, st.y, st.z], 1)
    A = np.array([[40.0, 10.0, 0.0], [10.0, -20.0, 5.0], [0.0, 5.0, -20.0]])
    V = X @ A.T
    st.vx[:], st.vy[:], st.vz[:] = V[:, 0], V[:, 1], V[:, 2]
    st.E[:] = 0.5 * (V * V).sum(axis=1)                # e = 0, S = 0, rho = rho0: sigma = 0
    M = _lattice_moment(s.h, s.dx)
    m = M[0, 0]
    assert np.abs(M - m * np.eye(3)).max() < 1e-12 * m
    inn = _interior(s, margin=4)
    assert inn.sum() == 27
    h0 = _heating(s, st, 0)[inn]
    h1 = _heating(s, st, 1)[inn]
    assert (h0 > 0).all()                              # first order: numerical heating everywhere
    assert np.abs(h1 / h0 - (1.0 - m)).max() <= 1e-9


def test_volume_rate_and_velocity_gradient_keep_the_particle_velocities():
    # the transport velocity is the particle velocity: the volume rate w_i sum w_j (v_j - v_i) . grad W
    # and the velocity gradient L of the stress rate do not see the reconstruction, bit for bit
    s, P, st = _state(n_side=8, jitter=0.01, walls=[(2, 0.0)])
    rng = np.random.default_rng(9)
    for f, a in (("vx", 20.0), ("vy", 20.0), ("vz", 20.0)):
        getattr(st, f)[:] = rng.normal(0, a, st.n)
    for f in ("sxx", "syy", "sxy", "sxz", "syz"):
        getattr(st, f)[:] = rng.normal(0, 3e7, st.n)
    st.szz[:] = -(st.sxx + st.syy)
    r1, _, _ = orc.rates(P, st)
    s.reconstruction = 0
    r0, _, _ = orc.rates(orc.params_of(s), st)
    assert (r1[:, 0] == r0[:, 0]).all()
    assert (r1[:, 6:] == r0[:, 6:]).all()
    assert np.abs(r1[:, 1:6] - r0[:, 1:6]).max() > 0     # the fluxes do change
