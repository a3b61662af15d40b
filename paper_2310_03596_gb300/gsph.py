"""Thin ctypes binding of libgsph (include/gsph.h): argument marshalling only.

Every step of the hot path runs in the CUDA library. PyTorch provides device buffers and streams
where the caller wants them (torch tensors on the context's GPU are passed by data pointer). If the
library is missing, load() raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import scenes

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgsph.so")

MAX_MAT, MAX_WALL, MAX_LABEL, NRATE = 4, 6, 16, 15
FP64, FP32_SPLIT = 0, 1

STATUS = {0: "ok", 1: "invalid argument", 2: "device out of memory", 3: "CUDA error",
          4: "particles left the bucket grid", 5: "bounded device wait timed out", 6: "no particles loaded",
          7: "invalid data found on the device"}
OK, INVALID_ARG, OOM, CUDA_ERROR, PARTICLE_LEFT_DOMAIN, DEVICE_TIMEOUT, NOT_READY, DEVICE_ERROR = range(8)

# gsph_field
FIELDS = ["x", "y", "z", "vx", "vy", "vz", "w", "m", "E", "sxx", "syy", "szz", "sxy", "sxz", "syz",
          "material", "label", "id", "hash", "comm_hash", "flag", "nreal", "nimage", "rates", "boundary", "h"]
FIELD = {name: k for k, name in enumerate(FIELDS)}
FIELD_DTYPE = {**{f: np.float64 for f in FIELDS[:15]}, "material": np.uint8, "label": np.uint8,
               "id": np.uint32, "hash": np.uint32, "comm_hash": np.uint32, "flag": np.uint8,
               "nreal": np.int32, "nimage": np.int32, "rates": np.float64, "boundary": np.uint32, "h": np.float64}


class GsphError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)} ({code})")
        self.code = code


class Material(C.Structure):
    _fields_ = [("rho0", C.c_double), ("K", C.c_double), ("G", C.c_double), ("Y", C.c_double),
                ("eos", C.c_int32), ("pad", C.c_int32), ("c0", C.c_double), ("s", C.c_double),
                ("gamma0", C.c_double), ("p_min", C.c_double)]


class Wall(C.Structure):
    _fields_ = [("axis", C.c_int32), ("pad", C.c_int32), ("pos", C.c_double)]


class Config(C.Structure):
    _fields_ = [("grid_lo", C.c_double * 3), ("grid_dims", C.c_int32 * 3), ("n_materials", C.c_int32),
                ("h", C.c_double), ("cfl", C.c_double), ("materials", Material * MAX_MAT),
                ("n_walls", C.c_int32), ("K", C.c_int32), ("walls", Wall * MAX_WALL),
                ("gravity", C.c_double * 3), ("alpha", C.c_double), ("swap_period", C.c_int32),
                ("precision", C.c_int32), ("device", C.c_int32), ("diagnostics", C.c_int32),
                ("overlap", C.c_int32), ("integrator", C.c_int32), ("reconstruction", C.c_int32),
                ("variable_h", C.c_int32)]


class ExchangeStats(C.Structure):
    _fields_ = [("step", C.c_int64), ("n", C.c_int64), ("K", C.c_int32), ("pad", C.c_int32),
                ("garbage", C.c_int64), ("boundary", C.c_int64 * MAX_LABEL), ("boundary_total", C.c_int64),
                ("exchange_fraction", C.c_double), ("record_bytes", C.c_int64),
                ("bytes_hash_broadcast", C.c_int64), ("bytes_boundary_broadcast", C.c_int64),
                ("bytes_swap", C.c_int64), ("swapped_last_pass", C.c_int64), ("swap_passes", C.c_int64),
                ("pairs_total", C.c_int64), ("kernel_launches", C.c_int64),
                ("cost", C.c_int64 * MAX_LABEL), ("cost_imbalance", C.c_double),
                ("dt_candidates", C.c_int64), ("dt_fp64_evaluations", C.c_int64), ("swap_fp64_hashes", C.c_int64)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("pad", "boundary", "cost")}
        d["boundary"] = list(self.boundary)[: self.K]
        d["cost"] = list(self.cost)[: self.K]
        return d


class AdjConfig(C.Structure):
    _fields_ = [("steps", C.c_int32), ("every", C.c_int32), ("n_obs", C.c_int64),
                ("obs_ids", C.POINTER(C.c_uint32)), ("dts", C.POINTER(C.c_double)),
                ("dts_out", C.POINTER(C.c_double)), ("J", C.POINTER(C.c_double)),
                ("want_gradient", C.c_int32), ("pad", C.c_int32)]


class Timings(C.Structure):
    _fields_ = [("hash_sort_ms", C.c_double), ("reorder_ms", C.c_double), ("swap_ms", C.c_double),
                ("comm_ms", C.c_double), ("interact_ms", C.c_double), ("steps", C.c_int64),
                ("interact_launches", C.c_int64), ("nbr_list_ms", C.c_double), ("pair_ms", C.c_double),
                ("local_ms", C.c_double), ("boundary_ms", C.c_double), ("halo_ms", C.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


EXPORTS = ["gsph_status_str", "gsph_create", "gsph_destroy", "gsph_set_particles", "gsph_put_field",
           "gsph_get_field", "gsph_step", "gsph_swap_now", "gsph_sync", "gsph_get_exchange_stats",
           "gsph_get_conserved", "gsph_get_dt", "gsph_get_sizes", "gsph_set_timing", "gsph_set_timing_ex",
           "gsph_get_timings",
           "gsph_radix_sort_workspace", "gsph_radix_sort_pairs", "gsph_radix_sort_pairs_noalloc",
           "gsph_set_dt", "gsph_adjoint_step", "gsph_state_bytes", "gsph_save_state", "gsph_load_state",
           "gsph_adjoint", "gsph_set_wait_limit", "gsph_debug_fail_alloc"]
SORT_NOALLOC_MAX_N = 1 << 20

_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Loads libgsph.so (built by paper_2310_03596_gb300.build). Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libgsph.so is not built ({path}); run paper_2310_03596_gb300.build.build()")
        L = C.CDLL(path)
        P, vp = C.POINTER, C.c_void_p
        L.gsph_status_str.argtypes = [C.c_int]
        L.gsph_status_str.restype = C.c_char_p
        L.gsph_create.argtypes = [P(Config), P(vp)]
        L.gsph_destroy.argtypes = [vp]
        L.gsph_destroy.restype = None
        L.gsph_set_particles.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp, C.c_int32, vp]
        L.gsph_put_field.argtypes = [vp, C.c_int, vp, C.c_int32, vp]
        L.gsph_get_field.argtypes = [vp, C.c_int, vp, C.c_int32, vp]
        L.gsph_step.argtypes = [vp, C.c_int32, vp]
        L.gsph_swap_now.argtypes = [vp, vp]
        L.gsph_sync.argtypes = [vp, vp]
        L.gsph_get_exchange_stats.argtypes = [vp, vp, P(ExchangeStats)]
        L.gsph_get_conserved.argtypes = [vp, vp, P(C.c_double)]
        L.gsph_get_dt.argtypes = [vp, vp, P(C.c_double)]
        L.gsph_get_sizes.argtypes = [vp, P(C.c_int64), P(C.c_int64)]
        L.gsph_set_timing.argtypes = [vp, C.c_int32]
        L.gsph_set_timing_ex.argtypes = [vp, C.c_int32, C.c_int32]
        L.gsph_get_timings.argtypes = [vp, P(Timings)]
        L.gsph_radix_sort_workspace.argtypes = [C.c_int64, C.c_int32]
        L.gsph_radix_sort_workspace.restype = C.c_size_t
        L.gsph_radix_sort_pairs.argtypes = [vp, vp, C.c_int64, C.c_int32, vp, C.c_size_t, vp]
        L.gsph_radix_sort_pairs_noalloc.argtypes = [vp, vp, C.c_int64, C.c_int32, vp]
        L.gsph_set_dt.argtypes = [vp, C.c_double, vp]
        L.gsph_adjoint_step.argtypes = [vp, vp, vp, C.c_double, P(C.c_double), vp]
        L.gsph_state_bytes.argtypes = [vp]
        L.gsph_state_bytes.restype = C.c_size_t
        L.gsph_save_state.argtypes = [vp, vp, C.c_size_t, C.c_int32, vp]
        L.gsph_load_state.argtypes = [vp, vp, C.c_size_t, C.c_int32, vp]
        L.gsph_adjoint.argtypes = [vp, P(AdjConfig), P(C.c_double), vp]
        L.gsph_set_wait_limit.argtypes = [vp, C.c_uint32, C.c_uint32]
        L.gsph_debug_fail_alloc.argtypes = [C.c_int32]
        L.gsph_debug_fail_alloc.restype = None
        _lib = L
        return L


def check(code: int, what: str, allow=(OK,)) -> int:
    if code not in allow:
        raise GsphError(code, what)
    return code


def config_from_scene(scene, precision: int = FP32_SPLIT, device: int = 0, diagnostics: bool = False,
                      overlap: bool = False) -> Config:
    c = Config()
    for a in range(3):
        c.grid_lo[a] = scene.grid_lo[a]
        c.grid_dims[a] = scene.grid_dims[a]
        c.gravity[a] = scene.gravity[a]
    c.n_materials = len(scene.materials)
    for k, (rho0, K, G, Y) in enumerate(scene.materials):
        eos, c0, sl, g0, pmin = scenes.material_eos(scene, k)
        c.materials[k] = Material(rho0, K, G, Y, eos, 0, c0, sl, g0, pmin)
    c.h = scene.h
    c.cfl = scene.cfl
    c.n_walls = len(scene.walls)
    for k, (axis, pos) in enumerate(scene.walls):
        c.walls[k] = Wall(axis, 0, pos)
    c.K = scene.K
    c.alpha = scene.alpha
    c.swap_period = scene.swap_period
    c.precision = precision
    c.device = device
    c.diagnostics = int(diagnostics)
    c.overlap = int(overlap)
    c.integrator = int(getattr(scene, "integrator", 0) or 0)
    c.reconstruction = int(getattr(scene, "reconstruction", 0) or 0)
    c.variable_h = int(getattr(scene, "variable_h", 0) or 0)
    return c


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


class Solver:
    """One libgsph context (one particle set on one GPU)."""

    def __init__(self, config: Config):
        self.L = load()
        self.cfg = config
        h = C.c_void_p()
        check(self.L.gsph_create(C.byref(config), C.byref(h)), "gsph_create")
        self.h = h
        self.n = 0

    @classmethod
    def from_scene(cls, scene, precision: int = FP32_SPLIT, device: int = 0, diagnostics: bool = False,
                   stream=None, overlap: bool = False) -> "Solver":
        s = cls(config_from_scene(scene, precision, device, diagnostics, overlap))
        s.set_particles(scene.pos, scene.vel, scene.vol, scene.material, scene.label, stream=stream)
        if getattr(scene, "variable_h", 0):
            s.put("h", np.asarray(scene.hp, dtype=np.float64), stream=stream)
        return s

    def close(self) -> None:
        if self.h:
            self.L.gsph_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------------------------- state
    def set_particles(self, pos, vel, vol, material, label, stream=None) -> None:
        arrs = [pos, vel, vol, material, label]
        if all(_is_torch(a) and a.is_cuda for a in arrs):
            for a in arrs:
                assert a.is_contiguous()
            ptrs = [a.data_ptr() for a in arrs]
            n = int(vol.shape[0])
            on_dev = 1
            keep = arrs
        else:
            keep = [np.ascontiguousarray(pos, np.float64), np.ascontiguousarray(vel, np.float64),
                    np.ascontiguousarray(vol, np.float64), np.ascontiguousarray(material, np.uint8),
                    np.ascontiguousarray(label, np.uint8)]
            ptrs = [a.ctypes.data for a in keep]
            n = int(keep[2].shape[0])
            on_dev = 0
        check(self.L.gsph_set_particles(self.h, n, *ptrs, on_dev, _stream_handle(stream)), "gsph_set_particles")
        self.n = n
        del keep

    def step(self, nsteps: int = 1, stream=None) -> None:
        check(self.L.gsph_step(self.h, int(nsteps), _stream_handle(stream)), "gsph_step")

    def swap_now(self, stream=None) -> None:
        check(self.L.gsph_swap_now(self.h, _stream_handle(stream)), "gsph_swap_now")

    def sync(self, stream=None) -> None:
        check(self.L.gsph_sync(self.h, _stream_handle(stream)), "gsph_sync")

    def _count(self, field: str) -> int:
        if field == "rates":
            return self.n * NRATE
        if field == "boundary":
            return int(self.exchange_stats()["boundary_total"])
        return self.n

    def get(self, field: str, stream=None, out: np.ndarray | None = None) -> np.ndarray:
        """Copies one field to host memory: a new numpy array, or `out` (e.g. a pinned buffer)."""
        cnt = self._count(field)
        if out is None:
            buf = np.empty(max(cnt, 1), FIELD_DTYPE[field])
        else:
            buf = out.reshape(-1)
            assert buf.dtype == FIELD_DTYPE[field] and buf.size >= cnt and buf.flags.c_contiguous
        check(self.L.gsph_get_field(self.h, FIELD[field], buf.ctypes.data, 0, _stream_handle(stream)),
              f"gsph_get_field({field})")
        if out is not None:
            return out
        buf = buf[:cnt]
        return buf.reshape(self.n, NRATE) if field == "rates" else buf

    def get_into(self, field: str, dst, stream=None) -> None:
        """Copies one field into a device tensor (torch, on the context's GPU)."""
        check(self.L.gsph_get_field(self.h, FIELD[field], dst.data_ptr(), 1, _stream_handle(stream)),
              f"gsph_get_field({field})")

    def put(self, field: str, values, stream=None) -> None:
        if _is_torch(values) and values.is_cuda:
            check(self.L.gsph_put_field(self.h, FIELD[field], values.data_ptr(), 1, _stream_handle(stream)),
                  f"gsph_put_field({field})")
            return
        a = np.ascontiguousarray(values, FIELD_DTYPE[field])
        assert a.shape[0] == self.n
        check(self.L.gsph_put_field(self.h, FIELD[field], a.ctypes.data, 0, _stream_handle(stream)),
              f"gsph_put_field({field})")

    def put_state(self, d: dict, stream=None) -> None:
        for f in FIELDS[:18]:
            if f in d:
                self.put(f, d[f], stream)

    def state(self, stream=None) -> dict:
        d = {f: self.get(f, stream) for f in FIELDS[:18]}
        if self.cfg.variable_h:
            d["h"] = self.get("h", stream)
        return d

    # ---------------------------------------------------------------------------- queries
    def exchange_stats(self, stream=None) -> dict:
        st = ExchangeStats()
        check(self.L.gsph_get_exchange_stats(self.h, _stream_handle(stream), C.byref(st)), "gsph_get_exchange_stats",
              allow=(OK, PARTICLE_LEFT_DOMAIN))
        return st.as_dict()

    def conserved(self, stream=None) -> np.ndarray:
        out = (C.c_double * 6)()
        check(self.L.gsph_get_conserved(self.h, _stream_handle(stream), out), "gsph_get_conserved")
        return np.array(out[:])

    def dt(self, stream=None) -> float:
        v = C.c_double()
        check(self.L.gsph_get_dt(self.h, _stream_handle(stream), C.byref(v)), "gsph_get_dt")
        return v.value

    def sizes(self):
        n, c = C.c_int64(), C.c_int64()
        check(self.L.gsph_get_sizes(self.h, C.byref(n), C.byref(c)), "gsph_get_sizes")
        return n.value, c.value

    def set_dt(self, dt: float, stream=None) -> None:
        """Time step of the next step (replay of a recorded schedule)."""
        check(self.L.gsph_set_dt(self.h, float(dt), _stream_handle(stream)), "gsph_set_dt")

    def adjoint_step(self, lam_next, lam_prev, dt: float, stream=None):
        """Reverse-mode step at the current state (FP64 context with diagnostics): lam_prev = dJ/dy_n
        from lam_next = dJ/dy_{n+1} (device tensors, 15 x n float64, field-major). Returns the step's
        direct (dJ/dY, dJ/dG) contributions."""
        g = (C.c_double * 2)()
        check(self.L.gsph_adjoint_step(self.h, lam_next.data_ptr(), lam_prev.data_ptr(), float(dt), g,
                                       _stream_handle(stream)), "gsph_adjoint_step")
        return g[0], g[1]

    # ------------------------------------------------------------------ checkpoint / resume
    def state_bytes(self) -> int:
        return int(self.L.gsph_state_bytes(self.h))

    def save_state(self, out=None, stream=None):
        """The context's state as a blob: a new host uint8 array, or `out` (a host array or a device
        tensor of at least state_bytes() bytes)."""
        nb = self.state_bytes()
        if out is None:
            out = np.empty(nb, np.uint8)
        if _is_torch(out) and out.is_cuda:
            assert out.is_contiguous() and out.numel() * out.element_size() >= nb
            check(self.L.gsph_save_state(self.h, out.data_ptr(), nb, 1, _stream_handle(stream)), "gsph_save_state")
        else:
            assert out.flags.c_contiguous and out.nbytes >= nb
            check(self.L.gsph_save_state(self.h, out.ctypes.data, nb, 0, _stream_handle(stream)), "gsph_save_state")
        return out

    def load_state(self, blob, stream=None) -> None:
        if _is_torch(blob) and blob.is_cuda:
            assert blob.is_contiguous()
            nb = blob.numel() * blob.element_size()
            check(self.L.gsph_load_state(self.h, blob.data_ptr(), nb, 1, _stream_handle(stream)), "gsph_load_state")
        else:
            a = np.ascontiguousarray(blob)
            check(self.L.gsph_load_state(self.h, a.ctypes.data, a.nbytes, 0, _stream_handle(stream)), "gsph_load_state")
        self.n = self.sizes()[0]

    def adjoint(self, steps: int, every: int, obs_ids, dts=None, want_gradient: bool = True, stream=None):
        """gsph_adjoint: J = mean z velocity of the particles obs_ids after `steps` steps from the current
        state and, with want_gradient, (dJ/dY, dJ/dG, dJ/dv0) by the checkpointed reverse sweep. dts: the
        time-step schedule (steps values), or None for the run's own CFL steps, held fixed. Returns
        (J, grad or None, the schedule used)."""
        ids = np.ascontiguousarray(obs_ids, np.uint32)
        a = AdjConfig()
        a.steps, a.every, a.n_obs = int(steps), int(every), int(ids.size)
        a.obs_ids = ids.ctypes.data_as(C.POINTER(C.c_uint32))
        dv = None
        if dts is not None:
            dv = np.ascontiguousarray(dts, np.float64)
            assert dv.size == steps
            a.dts = dv.ctypes.data_as(C.POINTER(C.c_double))
        out = np.empty(int(steps), np.float64)
        a.dts_out = out.ctypes.data_as(C.POINTER(C.c_double))
        J = C.c_double()
        a.J = C.pointer(J)
        a.want_gradient = int(bool(want_gradient))
        g = (C.c_double * 3)()
        check(self.L.gsph_adjoint(self.h, C.byref(a), g, _stream_handle(stream)), "gsph_adjoint")
        return J.value, (tuple(g[:]) if want_gradient else None), out

    def set_timing(self, max_steps: int, pair_only: bool = False) -> None:
        """Arms CUDA-event timing for up to max_steps steps: every phase, or (pair_only) only the events
        that bound the pair kernel, the other phases then reading 0."""
        check(self.L.gsph_set_timing_ex(self.h, int(max_steps), 1 if pair_only else 0), "gsph_set_timing_ex")

    def timings(self) -> dict:
        t = Timings()
        check(self.L.gsph_get_timings(self.h, C.byref(t)), "gsph_get_timings")
        return t.as_dict()


def _sort_args(keys, vals) -> int:
    """Checks the two tensors of a sort: 32-bit integer, contiguous, the same length, on the current
    CUDA device (the sort writes both in place). Returns their length."""
    import torch

    for t in (keys, vals):
        if not (_is_torch(t) and t.is_cuda and t.is_contiguous() and t.dtype in (torch.int32, torch.uint32)):
            raise ValueError("keys and vals must be contiguous 32-bit integer CUDA tensors")
        if t.device.index != torch.cuda.current_device():
            raise ValueError("keys and vals must be on the current CUDA device")
    if keys.numel() != vals.numel():
        raise ValueError("keys and vals must have the same length")
    return int(keys.numel())


def radix_sort_pairs(keys, vals, key_bits: int, stream=None) -> None:
    """Stable in-place sort of two uint32 device tensors (torch int32 views) by the low key_bits."""
    import torch

    L = load()
    n = _sort_args(keys, vals)
    ws_bytes = int(L.gsph_radix_sort_workspace(n, key_bits))
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=keys.device)
    check(L.gsph_radix_sort_pairs(keys.data_ptr(), vals.data_ptr(), n, key_bits, ws.data_ptr(), ws_bytes,
                                  _stream_handle(stream)), "gsph_radix_sort_pairs")


def radix_sort_pairs_noalloc(keys, vals, key_bits: int, stream=None) -> None:
    """The same sort with no allocation at all (library-owned fixed scratch, n <= SORT_NOALLOC_MAX_N),
    for callers that cannot allocate device memory. Calls that overlap on the GPU race."""
    L = load()
    n = _sort_args(keys, vals)
    check(L.gsph_radix_sort_pairs_noalloc(keys.data_ptr(), vals.data_ptr(), n, key_bits,
                                          _stream_handle(stream)), "gsph_radix_sort_pairs_noalloc")
