"""ctypes wrapper of the plain FP64 CPU oracle (oracle/gsph_oracle.cpp).

TEST INFRASTRUCTURE ONLY: only tests/, the smoke check and the benchmark's CPU-baseline leg import
this module. It never touches the CUDA library and the CUDA library never touches it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liborc.so")
SRC = os.path.join(HERE, "gsph_oracle.cpp")
NRATE = 15
MAX_MAT, MAX_WALL = 4, 6

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liborc.so (g++, FP contraction off)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(SRC),
                                                  os.path.getmtime(os.path.join(HERE, "gsph_oracle.h")))):
        return LIB_PATH
    tmp = LIB_PATH + f".{os.getpid()}.tmp"
    base = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, SRC]
    # the per-particle loops may use OpenMP host threads (orc_set_threads); without it they run on one
    if subprocess.call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL) != 0:
        subprocess.check_call(base)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Material(C.Structure):
    _fields_ = [("rho0", C.c_double), ("K", C.c_double), ("G", C.c_double), ("Y", C.c_double),
                ("eos", C.c_int32), ("pad", C.c_int32), ("c0", C.c_double), ("s", C.c_double),
                ("gamma0", C.c_double), ("p_min", C.c_double)]


class Wall(C.Structure):
    _fields_ = [("axis", C.c_int32), ("pad", C.c_int32), ("pos", C.c_double)]


class Params(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("dims", C.c_int32 * 3), ("nmat", C.c_int32),
                ("h", C.c_double), ("cfl", C.c_double), ("mat", Material * MAX_MAT),
                ("nwalls", C.c_int32), ("K", C.c_int32), ("wall", Wall * MAX_WALL),
                ("g", C.c_double * 3), ("alpha", C.c_double), ("integrator", C.c_int32), ("pad2", C.c_int32),
                ("reconstruction", C.c_int32), ("variable_h", C.c_int32)]


_DP = C.POINTER(C.c_double)
_U8P = C.POINTER(C.c_uint8)
_U32P = C.POINTER(C.c_uint32)


class StateC(C.Structure):
    _fields_ = ([("n", C.c_int64)] +
                [(f, _DP) for f in ("x", "y", "z", "vx", "vy", "vz", "w", "m", "E",
                                    "sxx", "syy", "szz", "sxy", "sxz", "syz")] +
                [("mat", _U8P), ("label", _U8P), ("id", _U32P), ("h", _DP)])


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER
            L.orc_hash.argtypes = [P(Params), C.c_int64, _DP, _DP, _DP, _U32P]
            L.orc_sort_order.argtypes = [C.c_int64, _U32P, P(C.c_int64)]
            L.orc_cell_ranges.argtypes = [C.c_int64, _U32P, C.c_int64, P(C.c_int64), P(C.c_int64)]
            for f in (L.orc_neighbours_brute, L.orc_neighbours_cells):
                f.argtypes = [P(Params), C.c_int64, _DP, _DP, _DP, C.c_int64, P(C.c_int32), P(C.c_int64), _DP]
                f.restype = C.c_int64
            L.orc_rates.argtypes = [P(Params), P(StateC), C.c_int64, P(C.c_int64), _DP, P(C.c_int32),
                                    P(C.c_int32)]
            L.orc_signal_speed.argtypes = [P(Params), P(StateC), C.c_int64]
            L.orc_signal_speed.restype = C.c_double
            L.orc_dt.argtypes = [P(Params), P(StateC)]
            L.orc_dt.restype = C.c_double
            L.orc_integrate.argtypes = [P(Params), P(StateC), _DP, C.c_double]
            L.orc_comm_hash.argtypes = [P(Params), C.c_int64, _U32P, _U8P, _U8P, _U32P, P(C.c_int64)]
            L.orc_boundary_lists.argtypes = [C.c_int64, _U8P, _U32P, C.c_uint32, C.c_int32,
                                             P(C.c_int64), P(C.c_int64)]
            L.orc_cg.argtypes = [P(Params), C.c_int64, _DP, _DP, _DP, _U8P, _U8P, C.c_int32, C.c_int32, _DP]
            L.orc_cg.restype = C.c_int64
            L.orc_balancing_hash.argtypes = [_DP, _DP, _DP]
            L.orc_balancing_hash.restype = C.c_int32
            L.orc_swap_pass.argtypes = [P(Params), C.c_int64, _DP, _DP, _DP, _U8P, _U32P, _U8P, P(C.c_int64)]
            L.orc_swap_pass.restype = C.c_int64
            L.orc_step.argtypes = [P(Params), P(StateC), C.c_int32, _U32P, _U32P, _U8P, P(C.c_int64),
                                   P(C.c_int32), P(C.c_int32), _DP, _DP]
            L.orc_kernel_w.argtypes = [C.c_double, C.c_double]
            L.orc_kernel_w.restype = C.c_double
            L.orc_kernel_dw.argtypes = [C.c_double, C.c_double]
            L.orc_kernel_dw.restype = C.c_double
            L.orc_riemann.argtypes = [C.c_double] * 6 + [_DP]
            L.orc_gradients.argtypes = [P(Params), P(StateC), _DP]
            L.orc_forward_gradient.argtypes = [P(Params), P(StateC), C.c_int32, _DP, C.c_int64, _U32P, _DP]
            L.orc_forward_gradient.restype = C.c_double
            L.orc_flops_per_pair.argtypes = []
            L.orc_flops_per_pair.restype = C.c_int64
            L.orc_set_threads.argtypes = [C.c_int32]
            L.orc_set_threads.restype = C.c_int32
            L.orc_set_threads(1)
            _lib = L
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _material_eos(scene, k: int):
    """(eos, c0, s, gamma0, p_min) of material k of a scene: its Mie-Gruneisen constants when given,
    else the linear EOS; the pressure cut-off, else none."""
    eos = getattr(scene, "eos", None)
    pmin = getattr(scene, "p_min", None)
    mg = eos[k] if eos is not None and k < len(eos) else None
    cut = pmin[k] if pmin is not None and k < len(pmin) and pmin[k] is not None else -np.inf
    if mg is None:
        return 0, 0.0, 0.0, 0.0, float(cut)
    c0, sl, g0 = mg
    return 1, float(c0), float(sl), float(g0), float(cut)


def params_of(scene) -> Params:
    """Oracle parameter block from a scene description (see paper_2310_03596_gb300.scenes)."""
    p = Params()
    for a in range(3):
        p.lo[a] = scene.grid_lo[a]
        p.dims[a] = scene.grid_dims[a]
        p.g[a] = scene.gravity[a]
    p.nmat = len(scene.materials)
    for k, (rho0, K, G, Y) in enumerate(scene.materials):
        eos, c0, sl, g0, pmin = _material_eos(scene, k)
        p.mat[k] = Material(rho0, K, G, Y, eos, 0, c0, sl, g0, pmin)
    p.h = scene.h
    p.cfl = scene.cfl
    p.integrator = int(getattr(scene, "integrator", 0) or 0)
    p.reconstruction = int(getattr(scene, "reconstruction", 0) or 0)
    p.variable_h = int(getattr(scene, "variable_h", 0) or 0)
    p.nwalls = len(scene.walls)
    for k, (axis, pos) in enumerate(scene.walls):
        p.wall[k] = Wall(axis, 0, pos)
    p.K = scene.K
    p.alpha = scene.alpha
    return p


FIELDS = ("x", "y", "z", "vx", "vy", "vz", "w", "m", "E", "sxx", "syy", "szz", "sxy", "sxz", "syz")


class OracleState:
    """FP64 SoA particle state owned by numpy; the layout the oracle's C functions read."""

    def __init__(self, n: int):
        self.n = n
        for f in FIELDS:
            setattr(self, f, np.zeros(n))
        self.mat = np.zeros(n, np.uint8)
        self.label = np.zeros(n, np.uint8)
        self.id = np.arange(n, dtype=np.uint32)
        self.h = None          # per-particle smoothing lengths (variable h), else None

    @classmethod
    def from_scene(cls, scene) -> "OracleState":
        s = cls(scene.n)
        s.x[:], s.y[:], s.z[:] = scene.pos[:, 0], scene.pos[:, 1], scene.pos[:, 2]
        s.vx[:], s.vy[:], s.vz[:] = scene.vel[:, 0], scene.vel[:, 1], scene.vel[:, 2]
        s.w[:] = scene.vol
        rho0 = np.array([m[0] for m in scene.materials])[scene.material]
        s.m[:] = rho0 * scene.vol
        s.E[:] = 0.5 * ((s.vx * s.vx + s.vy * s.vy) + s.vz * s.vz)
        s.mat[:] = scene.material
        s.label[:] = scene.label
        if getattr(scene, "variable_h", 0):
            s.h = np.array(scene.hp, dtype=np.float64)
        return s

    @classmethod
    def from_arrays(cls, d: dict) -> "OracleState":
        n = len(d["x"])
        s = cls(n)
        for f in FIELDS + ("mat", "label", "id"):
            getattr(s, f)[:] = d[f] if f in d else d["material"]
        if d.get("h") is not None:
            s.h = np.array(d["h"], dtype=np.float64)
        return s

    def arrays(self) -> dict:
        d = {f: getattr(self, f).copy() for f in FIELDS + ("mat", "label", "id")}
        if self.h is not None:
            d["h"] = self.h.copy()
        return d

    def copy(self) -> "OracleState":
        return OracleState.from_arrays(self.arrays())

    def permute(self, perm: np.ndarray) -> None:
        for f in FIELDS + ("mat", "label", "id"):
            setattr(self, f, np.ascontiguousarray(getattr(self, f)[perm]))
        if self.h is not None:
            self.h = np.ascontiguousarray(self.h[perm])

    def cstruct(self) -> StateC:
        for f in FIELDS:
            setattr(self, f, np.ascontiguousarray(getattr(self, f), dtype=np.float64))
        c = StateC()
        c.n = self.n
        for f in FIELDS:
            setattr(c, f, _ptr(getattr(self, f), C.c_double))
        c.mat = _ptr(self.mat, C.c_uint8)
        c.label = _ptr(self.label, C.c_uint8)
        c.id = _ptr(self.id, C.c_uint32)
        if self.h is not None:
            self.h = np.ascontiguousarray(self.h, dtype=np.float64)
            c.h = _ptr(self.h, C.c_double)
        return c


def hash_keys(P: Params, x, y, z) -> np.ndarray:
    x, y, z = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z))
    key = np.empty(len(x), np.uint32)
    lib().orc_hash(C.byref(P), len(x), _ptr(x, C.c_double), _ptr(y, C.c_double), _ptr(z, C.c_double),
                   _ptr(key, C.c_uint32))
    return key


def eos(P: Params, mat: int, rho: float, e: float):
    """(p, bulk sound speed squared) of material mat at density rho and specific internal energy e."""
    p, cb2 = C.c_double(), C.c_double()
    lib().orc_eos(C.byref(P), C.c_int32(int(mat)), C.c_double(rho), C.c_double(e), C.byref(p), C.byref(cb2))
    return p.value, cb2.value


def sort_order(key: np.ndarray) -> np.ndarray:
    key = np.ascontiguousarray(key, dtype=np.uint32)
    perm = np.empty(len(key), np.int64)
    lib().orc_sort_order(len(key), _ptr(key, C.c_uint32), _ptr(perm, C.c_int64))
    return perm


def cell_ranges(sorted_key: np.ndarray, ncell: int):
    sorted_key = np.ascontiguousarray(sorted_key, dtype=np.uint32)
    st = np.empty(ncell, np.int64)
    en = np.empty(ncell, np.int64)
    lib().orc_cell_ranges(len(sorted_key), _ptr(sorted_key, C.c_uint32), ncell, _ptr(st, C.c_int64),
                          _ptr(en, C.c_int64))
    return st, en


def neighbours(P: Params, x, y, z, cap: int = 256, brute: bool = False, h=None):
    """Neighbour lists (each row sorted) and counts; image neighbours encoded as j + n (1 + wall).
    h: per-particle smoothing lengths (support (h_i + h_j)^2), or None for the uniform 2h."""
    x, y, z = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z))
    hp = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
    n = len(x)
    cnt = np.zeros(n, np.int32)
    lst = np.full((n, cap), -1, np.int64)
    f = lib().orc_neighbours_brute if brute else lib().orc_neighbours_cells
    mx = f(C.byref(P), n, _ptr(x, C.c_double), _ptr(y, C.c_double), _ptr(z, C.c_double), cap,
           _ptr(cnt, C.c_int32), _ptr(lst, C.c_int64), None if hp is None else _ptr(hp, C.c_double))
    if mx > cap:
        raise ValueError(f"neighbour cap {cap} exceeded ({mx})")
    return cnt, lst


def rates(P: Params, st: OracleState, subset=None):
    n = st.n
    out = np.zeros((n, NRATE))
    nr = np.zeros(n, np.int32)
    ni = np.zeros(n, np.int32)
    cs = st.cstruct()
    if subset is None:
        lib().orc_rates(C.byref(P), C.byref(cs), 0, None, _ptr(out, C.c_double), _ptr(nr, C.c_int32),
                        _ptr(ni, C.c_int32))
    else:
        sub = np.ascontiguousarray(subset, dtype=np.int64)
        lib().orc_rates(C.byref(P), C.byref(cs), len(sub), _ptr(sub, C.c_int64), _ptr(out, C.c_double),
                        _ptr(nr, C.c_int32), _ptr(ni, C.c_int32))
    return out, nr, ni


def signal_speed(P: Params, st: OracleState) -> np.ndarray:
    """FP64 signal speed c + |v| of every particle."""
    cs = st.cstruct()
    return np.array([lib().orc_signal_speed(C.byref(P), C.byref(cs), i) for i in range(st.n)])


def dt(P: Params, st: OracleState) -> float:
    cs = st.cstruct()
    return lib().orc_dt(C.byref(P), C.byref(cs))


def integrate(P: Params, st: OracleState, r: np.ndarray, dt_: float) -> None:
    r = np.ascontiguousarray(r, dtype=np.float64)
    cs = st.cstruct()
    lib().orc_integrate(C.byref(P), C.byref(cs), _ptr(r, C.c_double), dt_)


def comm_hash(P: Params, key: np.ndarray, label: np.ndarray):
    key = np.ascontiguousarray(key, dtype=np.uint32)
    label = np.ascontiguousarray(label, dtype=np.uint8)
    n = len(key)
    flag = np.zeros(n, np.uint8)
    comm = np.zeros(n, np.uint32)
    cnt = np.zeros(P.K, np.int64)
    lib().orc_comm_hash(C.byref(P), n, _ptr(key, C.c_uint32), _ptr(label, C.c_uint8),
                        _ptr(flag, C.c_uint8), _ptr(comm, C.c_uint32), _ptr(cnt, C.c_int64))
    return flag, comm, cnt


def boundary_lists(label: np.ndarray, comm: np.ndarray, garbage: int, K: int):
    label = np.ascontiguousarray(label, dtype=np.uint8)
    comm = np.ascontiguousarray(comm, dtype=np.uint32)
    n = len(label)
    off = np.zeros(K + 1, np.int64)
    out = np.zeros(max(n, 1), np.int64)
    lib().orc_boundary_lists(n, _ptr(label, C.c_uint8), _ptr(comm, C.c_uint32), garbage, K,
                             _ptr(off, C.c_int64), _ptr(out, C.c_int64))
    return off, out[: off[K]]


def cg(P: Params, x, y, z, label, mat, lab: int, material: int = -1):
    x, y, z = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z))
    label = np.ascontiguousarray(label, dtype=np.uint8)
    mat = np.ascontiguousarray(mat, dtype=np.uint8)
    out = np.zeros(3)
    cnt = lib().orc_cg(C.byref(P), len(x), _ptr(x, C.c_double), _ptr(y, C.c_double), _ptr(z, C.c_double),
                       _ptr(label, C.c_uint8), _ptr(mat, C.c_uint8), lab, material, _ptr(out, C.c_double))
    return out, cnt


def balancing_hash(own, oth, p) -> int:
    own, oth, p = (np.ascontiguousarray(a, dtype=np.float64) for a in (own, oth, p))
    return int(lib().orc_balancing_hash(_ptr(own, C.c_double), _ptr(oth, C.c_double), _ptr(p, C.c_double)))


def swap_pass(P: Params, st: OracleState):
    """One swap-heuristic pass on st (labels changed in place). Returns (moved, per-pair counts)."""
    sw = np.zeros(P.K * P.K, np.int64)
    st.label = np.ascontiguousarray(st.label)
    tot = lib().orc_swap_pass(C.byref(P), st.n, _ptr(st.x, C.c_double), _ptr(st.y, C.c_double),
                              _ptr(st.z, C.c_double), _ptr(st.mat, C.c_uint8), _ptr(st.id, C.c_uint32),
                              _ptr(st.label, C.c_uint8), _ptr(sw, C.c_int64))
    return int(tot), sw.reshape(P.K, P.K)


def step(P: Params, st: OracleState, do_swap: bool = False, want_rates: bool = False, dt: float = 0.0) -> dict:
    """One full step in the paper's order; st is replaced by the new state in sorted order. dt > 0
    fixes the time step (else the CFL step)."""
    n = st.n
    key = np.zeros(n, np.uint32)
    comm = np.zeros(n, np.uint32)
    flag = np.zeros(n, np.uint8)
    cnt = np.zeros(P.K, np.int64)
    nr = np.zeros(n, np.int32)
    ni = np.zeros(n, np.int32)
    r = np.zeros((n, NRATE)) if want_rates else None
    dtv = np.array([float(dt)])
    cs = st.cstruct()
    lib().orc_step(C.byref(P), C.byref(cs), int(do_swap), _ptr(key, C.c_uint32), _ptr(comm, C.c_uint32),
                   _ptr(flag, C.c_uint8), _ptr(cnt, C.c_int64), _ptr(nr, C.c_int32), _ptr(ni, C.c_int32),
                   _ptr(r, C.c_double) if r is not None else None, _ptr(dtv, C.c_double))
    return {"key": key, "comm": comm, "flag": flag, "count": cnt, "nreal": nr, "nimage": ni,
            "rates": r, "dt": float(dtv[0])}


def set_threads(n: int) -> int:
    """Host threads of the oracle's per-particle loops (1 by default); returns the count in effect."""
    return int(lib().orc_set_threads(int(n)))


def flops_per_pair() -> int:
    """+, -, *, / and sqrt of one ordered pair (flux and one end's accumulation), counted by the oracle."""
    return int(lib().orc_flops_per_pair())


def kernel_w(r: float, h: float) -> float:
    return lib().orc_kernel_w(r, h)


def kernel_dw(r: float, h: float) -> float:
    return lib().orc_kernel_dw(r, h)


def gradients(P: Params, st: OracleState) -> np.ndarray:
    """MUSCL gradients (n, 27): grad v row-major, then d sigma_c/dx_b for c = xx yy zz xy xz yz."""
    out = np.zeros((st.n, 27))
    cs = st.cstruct()
    lib().orc_gradients(C.byref(P), C.byref(cs), _ptr(out, C.c_double))
    return out


def riemann(uL, uR, tL, tR, ZL, ZR):
    out = np.zeros(2)
    lib().orc_riemann(uL, uR, tL, tR, ZL, ZR, _ptr(out, C.c_double))
    return float(out[0]), float(out[1])


def forward_gradient(P: Params, st: OracleState, dts, obs_id):
    dts = np.ascontiguousarray(dts, dtype=np.float64)
    obs = np.ascontiguousarray(obs_id, dtype=np.uint32)
    g = np.zeros(3)
    cs = st.cstruct()
    J = lib().orc_forward_gradient(C.byref(P), C.byref(cs), len(dts), _ptr(dts, C.c_double), len(obs),
                                   _ptr(obs, C.c_uint32), _ptr(g, C.c_double))
    return J, g
