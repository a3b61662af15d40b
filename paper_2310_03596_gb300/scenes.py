"""Seeded synthetic particle scenes for the impact and collapse workloads.

This module is the one piece shared by the CPU oracle's tests and the CUDA path. It builds, from a
seed, what a user hands the solver at initialisation: particle positions, velocities, volumes,
material ids and ownership labels, plus the fixed bucket grid, walls and materials of the scene.
It holds none of the method's arithmetic (no hashing, sorting, fluxes, integration or balancing).

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; the finaliser constants are Vigna's published ones), evaluated per
particle as a counter-based generator: draw k of particle `id` is mix(seed ^ (id * GOLDEN) +
(k + 1) * GOLDEN). Draws 0-2 jitter the three axes, draw 3 picks a random label.

Workloads (sizes as stated by the workload definitions; dx lattice spacing, h = 1.3 dx):
  cube_impact       16^3 aluminium cube, dx 1 mm, -100 m/s onto a wall at z = 0, one label
  taylor_bar        aluminium rod r 5 mm x 40 mm, dx 0.125 mm (1.61 M), 200 m/s onto a wall, K = 4
  projectile_plate  steel sphere r 5 mm at 1000 m/s onto an aluminium plate 60x60x10 mm, dx 0.2 mm,
                    K = 8 equal-count x-slabs, two materials
  collapse_block    aluminium block 0.4 x 0.2 x 0.1 m at dx 0.5 mm (64 M) on a floor, gravity, K = 16
  hvi_bead_plate    aluminium bead r 1.5 mm at 4.05 km/s, 32 degrees from the normal, onto a 2 mm
                    aluminium plate (Sec. IV); Mie-Gruneisen EOS with a spall cut-off, K = 4 x-slabs
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Materials: (rho0 kg/m^3, bulk modulus K Pa, shear modulus G Pa, yield stress Y Pa)
ALUMINIUM = (2700.0, 70.0e9, 26.0e9, 300.0e6)
STEEL = (7850.0, 160.0e9, 80.0e9, 1.0e9)

# Aluminium for the hypervelocity example (Sec. IV names Johnson-Cook in its elastic perfectly plastic
# limit with a Mie-Gruneisen EOS and a spall cut-off pressure, without values). These are inputs, the
# published constants of 6061-T6 aluminium (Steinberg's tables): rho0, c0, s, gamma0, G, and a yield
# stress and spall cut-off of that alloy. K = rho0 c0^2 (only the linear EOS would use it).
AL6061_RHO0, AL6061_C0, AL6061_S, AL6061_GAMMA0 = 2703.0, 5240.0, 1.40, 1.97
AL6061 = (AL6061_RHO0, AL6061_RHO0 * AL6061_C0 ** 2, 27.6e9, 290.0e6)
AL6061_P_MIN = -1.2e9


def splitmix64_draw(seed: int, ids: np.ndarray, k: int) -> np.ndarray:
    """Draw number k (0-based) of the counter-based SplitMix64 stream of each particle id."""
    with np.errstate(over="ignore"):
        s = np.uint64(seed) ^ (ids.astype(np.uint64) * GOLDEN)
        z = s + np.uint64(k + 1) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def unit_double(z: np.ndarray) -> np.ndarray:
    """Top 53 bits of a 64-bit draw as a double in [0, 1)."""
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclasses.dataclass
class Scene:
    """Initial particle set and the fixed setting it lives in (SoA, numpy, FP64 positions)."""

    name: str
    pos: np.ndarray            # (N, 3) float64
    vel: np.ndarray            # (N, 3) float64
    vol: np.ndarray            # (N,) float64
    material: np.ndarray       # (N,) uint8, index into materials
    label: np.ndarray          # (N,) uint8, ownership label in [0, K)
    materials: list            # [(rho0, K, G, Y), ...]
    h: float
    cfl: float
    grid_lo: tuple             # lower corner of the fixed bucket grid
    grid_dims: tuple           # buckets per axis; bucket side is 2h
    walls: list                # [(axis, position), ...] rigid mirror planes
    gravity: tuple
    K: int
    swap_period: int
    alpha: float
    steps: int
    dx: float
    eos: list = None           # per material: None (linear, K) or (c0, s, gamma0) Mie-Gruneisen
    p_min: list = None         # per material: pressure cut-off (Pa, <= 0) or None
    hp: np.ndarray = None      # (N,) per-particle smoothing lengths (variable_h = 1); h is their maximum
    variable_h: int = 0

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _jitter(pos: np.ndarray, ids: np.ndarray, seed: int, amp: float) -> np.ndarray:
    out = pos.copy()
    for ax in range(3):
        u = unit_double(splitmix64_draw(seed, ids, ax))
        out[:, ax] += amp * (2.0 * u - 1.0)
    return out


def _random_labels(ids: np.ndarray, seed: int, K: int) -> np.ndarray:
    z = splitmix64_draw(seed, ids, 3)
    return ((z >> np.uint64(32)) % np.uint64(K)).astype(np.uint8)


def _grid_around(pos: np.ndarray, h: float, margin_lo, margin_hi):
    cell = 2.0 * h
    lo = pos.min(axis=0) - np.asarray(margin_lo, dtype=np.float64)
    hi = pos.max(axis=0) + np.asarray(margin_hi, dtype=np.float64)
    dims = tuple(int(math.ceil((hi[a] - lo[a]) / cell)) for a in range(3))
    return tuple(float(v) for v in lo), dims


def _lattice(nx: int, ny: int, nz: int, dx: float, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Cell-centred lattice points origin + (i + 1/2) dx, x fastest."""
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    p = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64)
    return (p + 0.5) * dx + np.asarray(origin, dtype=np.float64)


def cube_impact(n_side: int = 16, dx: float = 1.0e-3, seed: int = 0, speed: float = 100.0,
                jitter: float = 0.01, steps: int = 10, K: int = 1) -> Scene:
    """Elastic-plastic aluminium cube falling at `speed` onto a rigid wall z = 0 it touches."""
    h = 1.3 * dx
    pos = _lattice(n_side, n_side, n_side, dx)
    ids = np.arange(pos.shape[0], dtype=np.uint64)
    if jitter:
        pos = _jitter(pos, ids, seed, jitter * dx)
    n = pos.shape[0]
    vel = np.zeros((n, 3))
    vel[:, 2] = -speed
    lo, dims = _grid_around(pos, h, (4 * h, 4 * h, 4 * h), (4 * h, 4 * h, 4 * h))
    label = _random_labels(ids, seed, K) if K > 1 else np.zeros(n, np.uint8)
    return Scene("cube_impact", pos, vel, np.full(n, dx ** 3), np.zeros(n, np.uint8), label,
                 [ALUMINIUM], h, 0.3, lo, dims, [(2, 0.0)], (0.0, 0.0, 0.0), K, 1, 0.1, steps, dx)


def _graded(fine_xy, nz_fine, nz_coarse, dx, origin_xy, seed, jitter, keep=None):
    """Two-resolution lattice along z: spacing dx for z < nz_fine dx, 2 dx above; h_i = 1.3 spacing."""
    nxf, nyf = fine_xy
    pf = _lattice(nxf, nyf, nz_fine, dx, origin=(origin_xy[0], origin_xy[1], 0.0))
    pc = _lattice(nxf // 2, nyf // 2, nz_coarse, 2 * dx, origin=(origin_xy[0], origin_xy[1], nz_fine * dx))
    if keep is not None:
        pf, pc = pf[keep(pf)], pc[keep(pc)]
    pos = np.concatenate([pf, pc])
    spacing = np.concatenate([np.full(len(pf), dx), np.full(len(pc), 2 * dx)])
    ids = np.arange(pos.shape[0], dtype=np.uint64)
    if jitter:
        pos = pos + (_jitter(pos, ids, seed, 1.0) - pos) * (jitter * spacing)[:, None]
    return pos, spacing, ids


def graded_block(n_side: int = 8, nz_fine: int = 8, nz_coarse: int = 4, dx: float = 1.0e-3, seed: int = 0,
                 speed: float = 100.0, jitter: float = 0.01, K: int = 1, wall: bool = True) -> Scene:
    """Aluminium block of two particle sizes (Sec. V's varying particle sizes): an n_side^2 x nz_fine
    layer of spacing dx on the rigid wall z = 0, under an (n_side/2)^2 x nz_coarse layer of spacing 2 dx,
    h_i = 1.3 x the particle's spacing, falling at `speed`."""
    pos, spacing, ids = _graded((n_side, n_side), nz_fine, nz_coarse, dx, (0.0, 0.0), seed, jitter)
    n = pos.shape[0]
    hp = 1.3 * spacing
    h = float(hp.max())
    vel = np.zeros((n, 3))
    vel[:, 2] = -speed
    lo, dims = _grid_around(pos, h, (4 * h, 4 * h, 4 * h), (4 * h, 4 * h, 4 * h))
    label = _random_labels(ids, seed, K) if K > 1 else np.zeros(n, np.uint8)
    sc = Scene("graded_block", pos, vel, spacing ** 3, np.zeros(n, np.uint8), label, [ALUMINIUM], h, 0.3, lo,
               dims, [(2, 0.0)] if wall else [], (0.0, 0.0, 0.0), K, 1, 0.1, 10, dx)
    sc.hp = hp
    sc.variable_h = 1
    return sc


def graded_bar(dx: float = 0.125e-3, radius: float = 5.0e-3, fine: float = 10.0e-3, length: float = 40.0e-3,
               speed: float = 200.0, seed: int = 1, K: int = 4, swap_period: int = 1, steps: int = 100) -> Scene:
    """The Taylor bar with two particle sizes: spacing dx over the impact end (z < fine), 2 dx over the
    rest of the rod, h_i = 1.3 x spacing, random labels."""
    nr = int(round(radius / dx))
    nzf = int(round(fine / dx))
    nzc = int(round((length - fine) / (2 * dx)))
    keep = lambda p: p[:, 0] ** 2 + p[:, 1] ** 2 <= radius ** 2
    pos, spacing, ids = _graded((2 * nr, 2 * nr), nzf, nzc, dx, (-nr * dx, -nr * dx), seed, 0.01, keep)
    n = pos.shape[0]
    hp = 1.3 * spacing
    h = float(hp.max())
    vel = np.zeros((n, 3))
    vel[:, 2] = -speed
    m = 4 * h
    lo, dims = _grid_around(pos, h, (m, m, m), (m, m, m))
    sc = Scene("graded_bar", pos, vel, spacing ** 3, np.zeros(n, np.uint8), _random_labels(ids, seed, K),
               [ALUMINIUM], h, 0.3, lo, dims, [(2, 0.0)], (0.0, 0.0, 0.0), K, swap_period, 0.1, steps, dx)
    sc.hp = hp
    sc.variable_h = 1
    return sc


def taylor_bar(dx: float = 0.125e-3, radius: float = 5.0e-3, length: float = 40.0e-3,
               speed: float = 200.0, seed: int = 1, K: int = 4, swap_period: int = 1,
               steps: int = 100) -> Scene:
    """Aluminium rod along z, base on the rigid wall z = 0, moving at -speed along z."""
    h = 1.3 * dx
    nr = int(round(radius / dx))
    nl = int(round(length / dx))
    pos = _lattice(2 * nr, 2 * nr, nl, dx, origin=(-nr * dx, -nr * dx, 0.0))
    keep = pos[:, 0] ** 2 + pos[:, 1] ** 2 <= radius ** 2
    pos = pos[keep]
    ids = np.arange(pos.shape[0], dtype=np.uint64)
    pos = _jitter(pos, ids, seed, 0.01 * dx)
    n = pos.shape[0]
    vel = np.zeros((n, 3))
    vel[:, 2] = -speed
    m = 4 * h
    lo, dims = _grid_around(pos, h, (m, m, m), (m, m, m))
    return Scene("taylor_bar", pos, vel, np.full(n, dx ** 3), np.zeros(n, np.uint8),
                 _random_labels(ids, seed, K), [ALUMINIUM], h, 0.3, lo, dims, [(2, 0.0)],
                 (0.0, 0.0, 0.0), K, swap_period, 0.1, steps, dx)


def projectile_plate(dx: float = 0.2e-3, radius: float = 5.0e-3, plate=(60.0e-3, 60.0e-3, 10.0e-3),
                     speed: float = 1000.0, seed: int = 2, K: int = 8, swap_period: int = 20,
                     steps: int = 500) -> Scene:
    """Steel sphere just above an aluminium plate (top face z = 0), moving at -speed along z."""
    h = 1.3 * dx
    px, py, pz = (int(round(v / dx)) for v in plate)
    plate_pos = _lattice(px, py, pz, dx, origin=(-px * dx / 2, -py * dx / 2, -pz * dx))
    nr = int(round(radius / dx))
    sph = _lattice(2 * nr, 2 * nr, 2 * nr, dx, origin=(-nr * dx, -nr * dx, -nr * dx))
    sph = sph[(sph ** 2).sum(axis=1) <= radius ** 2]
    sph[:, 2] += radius + dx
    pos = np.concatenate([plate_pos, sph])
    mat = np.concatenate([np.zeros(plate_pos.shape[0], np.uint8), np.ones(sph.shape[0], np.uint8)])
    ids = np.arange(pos.shape[0], dtype=np.uint64)
    pos = _jitter(pos, ids, seed, 0.01 * dx)
    n = pos.shape[0]
    vel = np.zeros((n, 3))
    vel[mat == 1, 2] = -speed
    # equal-count slabs along x
    order = np.argsort(pos[:, 0], kind="stable")
    label = np.empty(n, np.uint8)
    label[order] = (np.arange(n) * K // n).astype(np.uint8)
    m = 8.0e-3
    lo, dims = _grid_around(pos, h, (m, m, m), (m, m, m))
    return Scene("projectile_plate", pos, vel, np.full(n, dx ** 3), mat, label, [ALUMINIUM, STEEL],
                 h, 0.3, lo, dims, [], (0.0, 0.0, 0.0), K, swap_period, 0.1, steps, dx)


def collapse_block(dx: float = 0.5e-3, size=(0.4, 0.2, 0.1), seed: int = 4, K: int = 16,
                   swap_period: int = 10, steps: int = 200, gravity: float = 9.81) -> Scene:
    """Aluminium block at rest on a rigid floor z = 0 under gravity, random labels."""
    h = 1.3 * dx
    nx, ny, nz = (int(round(v / dx)) for v in size)
    pos = _lattice(nx, ny, nz, dx)
    ids = np.arange(pos.shape[0], dtype=np.uint64)
    pos = _jitter(pos, ids, seed, 0.01 * dx)
    n = pos.shape[0]
    m = 4 * h
    lo, dims = _grid_around(pos, h, (m, m, m), (m, m, m))
    return Scene("collapse_block", pos, np.zeros((n, 3)), np.full(n, dx ** 3), np.zeros(n, np.uint8),
                 _random_labels(ids, seed, K), [ALUMINIUM], h, 0.3, lo, dims, [(2, 0.0)],
                 (0.0, 0.0, -gravity), K, swap_period, 0.1, steps, dx)


def hvi_bead_plate(dx: float = 0.1e-3, radius: float = 1.5e-3, thickness: float = 2.0e-3,
                   side: float = 12.0e-3, speed: float = 4050.0, angle_deg: float = 32.0, seed: int = 5,
                   K: int = 4, swap_period: int = 10, steps: int = 200) -> Scene:
    """Aluminium bead just above an aluminium plate (top face z = 0), moving at `speed` tilted by
    `angle_deg` from the plate normal (the paper's hypervelocity example); Mie-Gruneisen EOS and spall
    cut-off for both."""
    h = 1.3 * dx
    px, pz = int(round(side / dx)), int(round(thickness / dx))
    plate = _lattice(px, px, pz, dx, origin=(-px * dx / 2, -px * dx / 2, -pz * dx))
    nr = int(round(radius / dx))
    bead = _lattice(2 * nr, 2 * nr, 2 * nr, dx, origin=(-nr * dx, -nr * dx, -nr * dx))
    bead = bead[(bead ** 2).sum(axis=1) <= radius ** 2]
    a = math.radians(angle_deg)
    bead[:, 0] -= (radius + dx) * math.tan(a)    # aimed at the plate centre
    bead[:, 2] += radius + dx
    pos = np.concatenate([plate, bead])
    ids = np.arange(pos.shape[0], dtype=np.uint64)
    pos = _jitter(pos, ids, seed, 0.01 * dx)
    n = pos.shape[0]
    vel = np.zeros((n, 3))
    nb = bead.shape[0]
    vel[n - nb:, 0] = speed * math.sin(a)
    vel[n - nb:, 2] = -speed * math.cos(a)
    order = np.argsort(pos[:, 0], kind="stable")
    label = np.empty(n, np.uint8)
    label[order] = (np.arange(n) * K // n).astype(np.uint8)
    m = 4.0e-3
    lo, dims = _grid_around(pos, h, (m, m, m), (m, m, m))
    return Scene("hvi_bead_plate", pos, vel, np.full(n, dx ** 3), np.zeros(n, np.uint8), label, [AL6061],
                 h, 0.3, lo, dims, [], (0.0, 0.0, 0.0), K, swap_period, 0.1, steps, dx,
                 eos=[(AL6061_C0, AL6061_S, AL6061_GAMMA0)], p_min=[AL6061_P_MIN])


def material_eos(scene, k: int):
    """(eos, c0, s, gamma0, p_min) of material k: 1 and its Mie-Gruneisen constants when the scene
    gives them, else 0 (linear EOS); the pressure cut-off, else -inf (none)."""
    mg = scene.eos[k] if scene.eos is not None and k < len(scene.eos) else None
    pm = scene.p_min[k] if scene.p_min is not None and k < len(scene.p_min) and scene.p_min[k] is not None \
        else -math.inf
    if mg is None:
        return 0, 0.0, 0.0, 0.0, float(pm)
    return 1, float(mg[0]), float(mg[1]), float(mg[2]), float(pm)


def adjoint_cube(n_side: int = 64, seed: int = 3, steps: int = 200) -> Scene:
    """The cube impact scaled up, used for the gradient workload."""
    s = cube_impact(n_side=n_side, seed=seed, steps=steps)
    s.name = "adjoint_cube"
    return s


WORKLOADS = {
    "hvi_bead_plate": hvi_bead_plate,
    "cube_impact": cube_impact,
    "taylor_bar": taylor_bar,
    "projectile_plate": projectile_plate,
    "adjoint_cube": adjoint_cube,
    "collapse_block": collapse_block,
}
