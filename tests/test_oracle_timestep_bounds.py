"""The CFL time step (Sec. II step g) is defined in FP64 (dt = cfl h / max(c + |v|)); the GPU step
evaluates the signal speed of every particle in FP32 with a running bound of the FP32 value's distance
from the FP64 one, and evaluates the FP64 sequence only for the particles whose interval reaches the
largest lower bound. These tests restate that FP32 interval in numpy float32 and check, over states from
rest to strong compression and tension, both equations of state and the branch point of the
Mie-Gruneisen reference curve, that the oracle's FP64 signal speed always lies inside it."""
import numpy as np

from oracle import orc
from paper_2310_03596_gb300 import scenes

f = np.float32
U = f(2.0 ** -24)
INF = f(np.inf)


class FE:
    """float32 value with a bound of its distance from the exact value (the kernel's running bound)."""

    def __init__(self, v, e):
        self.v, self.e = f(v), f(e)

    @staticmethod
    def inp(x):
        v = f(x)
        return FE(v, U * abs(v))

    def __add__(self, o):
        v = f(self.v + o.v)
        return FE(v, f(f(self.e + o.e) + U * abs(v)))

    def __sub__(self, o):
        v = f(self.v - o.v)
        return FE(v, f(f(self.e + o.e) + U * abs(v)))

    def __mul__(self, o):
        v = f(self.v * o.v)
        e = f(f(abs(self.v) * o.e) + f(abs(o.v) * self.e)) + f(self.e * o.e)
        return FE(v, f(e + U * abs(v)))

    def __truediv__(self, o):
        with np.errstate(all="ignore"):
            v = f(self.v / o.v)
            den = f(abs(o.v) - o.e)
            e = f(f(self.e + f(abs(v) * o.e)) / den) if den > 0 else INF
        return FE(v, f(e + U * abs(v)))

    def sqrt(self):
        v = f(np.sqrt(max(self.v, f(0))))
        r = f(np.sqrt(self.e))
        e = min(f(self.e / v), r) if v > 0 else r
        return FE(v, f(e + U * v))

    def scale(self, k):
        return FE(self.v * f(k), self.e * f(abs(k)))


def bounds(mat, m, w, vx, vy, vz, E):
    rho0, K, G = mat["rho0"], mat["K"], mat["G"]
    if mat.get("eos") is None:
        # linear EOS: non-negative quantities, relative error within 16 ulp (2^-20) of the FP32 value
        mf, wf, fx, fy, fz = f(m), f(w), f(vx), f(vy), f(vz)
        rho = f(mf / wf)
        v2 = f(f(f(fx * fx) + f(fy * fy)) + f(fz * fz))
        sv = f(f(np.sqrt(f(f(K + 4.0 * G / 3.0) / rho))) + f(np.sqrt(v2)))
        return f(sv * f(1 - 2.0 ** -20)), f(sv * f(1 + 2.0 ** -20))
    rho = FE.inp(m) / FE.inp(w)
    fx, fy, fz = FE.inp(vx), FE.inp(vy), FE.inp(vz)
    v2 = (fx * fx + fy * fy) + fz * fz
    vn = v2.sqrt()
    if True:
        c0, sl, g0 = mat["eos"]
        one = FE(1.0, 0.0)
        r0, C0, G0, SM1 = FE.inp(rho0), FE.inp(c0), FE.inp(g0), FE.inp(sl - 1.0)
        e = FE.inp(E) - v2.scale(0.5)
        mu = rho / r0 - one
        k0 = (r0 * C0) * C0
        q = one + mu
        r2 = r0.scale(2.0)
        gr = G0 * r0
        G43 = FE.inp(4.0 * G / 3.0)

        def branch(comp):
            if comp:
                D = one - SM1 * mu
                D2 = D * D
                pH = ((k0 * mu) * q) / D2
                a1 = (one + mu.scale(2.0)) * D
                a2 = (SM1.scale(2.0) * mu) * q
                dpH = (k0 * (a1 + a2)) / (D2 * D)
            else:
                pH, dpH = k0 * mu, k0
            eH = (pH * mu) / (r2 * q)
            deH = (((dpH * mu) * q) + pH) / ((r2 * q) * q)
            p = pH + gr * (e - eH)
            cb2 = (dpH - gr * deH) / r0 + (p * gr) / (rho * rho)
            cb2 = FE(max(cb2.v, f(0)), cb2.e)
            return (cb2 + G43 / rho).sqrt() + vn

        pos, neg = mu.v > mu.e, mu.v < -mu.e
        s1 = branch(not neg)
        s2 = s1 if (pos or neg) else branch(False)
    k = f(1.00390625)
    e1, e2 = f(s1.e * k), f(s2.e * k)
    lo = min(f(f(s1.v - e1) * f(1 - 2.0 ** -20)), f(f(s2.v - e2) * f(1 - 2.0 ** -20)))
    hi = max(f(f(s1.v + e1) * f(1 + 2.0 ** -20)), f(f(s2.v + e2) * f(1 + 2.0 ** -20)))
    return max(lo, f(0)), hi


def _check(scene, states):
    P = orc.params_of(scene)
    st = orc.OracleState(len(states))
    for i, (m, w, v, E) in enumerate(states):
        st.m[i], st.w[i] = m, w
        st.vx[i], st.vy[i], st.vz[i] = v
        st.E[i] = E
    sd = orc.signal_speed(P, st)
    rho0, K, G, _ = scene.materials[0]
    eos = getattr(scene, "eos", None)
    mat = {"rho0": rho0, "K": K, "G": G, "eos": eos[0] if eos else None}
    widths = []
    for i, (m, w, v, E) in enumerate(states):
        lo, hi = bounds(mat, m, w, *v, E)
        assert lo <= sd[i] <= hi, (i, m / w, v, E, lo, sd[i], hi)
        widths.append((hi - lo) / sd[i])
    return np.array(widths)


def test_linear_eos_interval_contains_fp64_signal_speed():
    s = scenes.cube_impact(n_side=2)
    rng = np.random.default_rng(5)
    rho0 = s.materials[0][0]
    states = []
    for _ in range(3000):
        w = 10.0 ** rng.uniform(-12, -6)
        m = rho0 * w * rng.choice([1.0, 1.0 + 1e-12, rng.uniform(0.5, 2.0)])
        v = rng.normal(0, 10.0 ** rng.uniform(-3, 3.5), 3) * rng.choice([0.0, 1.0])
        states.append((m, w, v, 0.0))
    wd = _check(s, states)
    assert wd.max() < 2.5e-6      # the interval is 2^-19 wide


def test_mie_gruneisen_interval_contains_fp64_signal_speed():
    s = scenes.hvi_bead_plate(dx=0.5e-3)
    rng = np.random.default_rng(6)
    rho0 = s.materials[0][0]
    states = []
    for _ in range(3000):
        w = 10.0 ** rng.uniform(-12, -8)
        ratio = rng.choice([1.0, 1.0 + 1e-9, 1.0 - 1e-9, 1.0 + 1e-6, rng.uniform(0.7, 1.6)])
        v = rng.normal(0, 10.0 ** rng.uniform(-2, 3.7), 3) * rng.choice([0.0, 1.0])
        E = 0.5 * float(v @ v) + rng.choice([0.0, 10.0 ** rng.uniform(2, 7)])
        states.append((rho0 * w * ratio, w, v, E))
    wd = _check(s, states)
    assert np.median(wd) < 1e-5
