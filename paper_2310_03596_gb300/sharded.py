"""Label-sharded multi-process data plane of the particle-decomposition method (Sec. II, Sec. III.A).

One process (rank) per ownership label: rank r holds the particles of label r, wherever they are in
space. A step follows the paper's order, with the exchanges as torch.distributed collectives:
  a. each rank hashes its own particles into the buckets of side 2h;
  swap heuristic (every P steps, Sec. III.A/B): the fixed-point Cg sums of every label (and type) are
     summed over the ranks; for each label pair in lexicographic order the two ranks compute their
     particles' balancing hashes, exchange their positive counts, select the n highest hashes (ties by
     persistent id) and exchange those particles (ownership moves with the label); the sums are
     updated by the moved particles;
  b. the per-bucket label masks are combined by an allreduce with bitwise OR (the hash broadcast);
  c. communication hash: a particle is an MGPU boundary particle when the 27 buckets around it hold
     another label;
  d. the boundary particles' records are all-gathered (variable counts) into each rank's halo;
  e-g. each rank's interaction engine evaluates its own particles against its own and the halo
     particles and integrates its own particles; the next time step is the minimum over the ranks.
The exchange bookkeeping (hash, masks, flags, fixed-point sums, balancing hashes, selection) runs as
torch tensor operations in FP64, each operation rounded once, so its integer results equal those of a
single-device run; the interaction and integration run in the engine (GpuEngine: libgsph). Works with
the gloo backend on CPU tensors and with NCCL on CUDA tensors.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

STATE = ("x", "y", "z", "vx", "vy", "vz", "w", "m", "E", "sxx", "syy", "szz", "sxy", "sxz", "syz")
INTS = ("mat", "label", "id")
HASH_MAX = 1000


class Grid:
    """The fixed bucket grid and the constants of the exchange (from a scene)."""

    def __init__(self, scene):
        self.lo = [float(v) for v in scene.grid_lo]
        self.dims = [int(v) for v in scene.grid_dims]
        self.cell = 2.0 * float(scene.h)
        self.ncell = self.dims[0] * self.dims[1] * self.dims[2]
        self.K = int(scene.K)
        self.alpha = float(scene.alpha)
        self.nmat = len(scene.materials)
        self.cfl, self.h = float(scene.cfl), float(scene.h)
        ext = [d * self.cell for d in self.dims]
        self.q_s = [4294967296.0 / e for e in ext]
        self.q_step = [e * 2.0 ** -32 for e in ext]


# --------------------------------------------------------------------------------- per-rank pieces
def bucket_keys(G: Grid, x, y, z):
    """Bucket hash: x-fastest linear index of floor((x - lo) / 2h) per axis; outside the grid (or NaN)
    the garbage value G.ncell."""
    out = torch.zeros(x.shape[0], dtype=torch.int64, device=x.device)
    ok = torch.ones(x.shape[0], dtype=torch.bool, device=x.device)
    mul = 1
    for a, v in enumerate((x, y, z)):
        t = (v - G.lo[a]) / G.cell
        inside = (t >= 0.0) & (t < float(G.dims[a]))
        ok &= inside
        c = torch.where(inside, t, torch.zeros_like(t)).to(torch.int64)   # truncation = floor for t >= 0
        out += c * mul
        mul *= G.dims[a]
    return torch.where(ok, out, torch.full_like(out, G.ncell))


def label_mask(G: Grid, key, label):
    """Per-bucket OR of (1 << label) over this rank's particles (int32, the garbage bucket dropped)."""
    mask = torch.zeros(G.ncell + 1, dtype=torch.int32, device=key.device)
    for lab in torch.unique(label).tolist():
        sel = label == lab
        occ = torch.bincount(key[sel], minlength=G.ncell + 1) > 0
        mask |= occ.to(torch.int32) << int(lab)
    return mask[: G.ncell]


def boundary_flags(G: Grid, key, label, mask):
    """MGPU boundary flag: the 27 buckets around the particle hold a label other than its own."""
    dx, dy, dz = G.dims
    inside = key < G.ncell
    k = torch.where(inside, key, torch.zeros_like(key))
    cx, cy, cz = k % dx, (k // dx) % dy, k // (dx * dy)
    acc = torch.zeros_like(k, dtype=torch.int32)
    for oz in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for ox in (-1, 0, 1):
                X, Y, Z = cx + ox, cy + oy, cz + oz
                ok = (X >= 0) & (X < dx) & (Y >= 0) & (Y < dy) & (Z >= 0) & (Z < dz)
                idx = torch.where(ok, X + dx * (Y + dy * Z), torch.zeros_like(X))
                acc |= torch.where(ok, mask[idx], torch.zeros_like(acc))
    other = acc & ~(torch.ones_like(acc) << label.to(torch.int32))
    return inside & (other != 0)


def fixed_point(G: Grid, v, a: int):
    """Cg fixed point of one axis: nearest integer (ties to even) to (v - lo) 2^32 / L, clamped to
    [0, 2^32 - 1], NaN to 0."""
    t = (v - G.lo[a]) * G.q_s[a]
    t = torch.where(torch.isnan(t), torch.zeros_like(t), t)
    q = torch.round(torch.clamp(t, 0.0, 4294967295.0))
    return q.to(torch.int64)


def balancing_hash(M, d, dn: float, ell: float, x, y, z):
    """Sec. III.A balancing hash in FP64 (each operation rounded): t = ((e0 d0 + e1 d1) + e2 d2) / |d|;
    0 for t <= 0, 1000 for t >= ell, else floor(1000 t / ell) clamped to [1, 1000]."""
    a0 = (x - M[0]) * d[0]
    a1 = (y - M[1]) * d[1]
    a2 = (z - M[2]) * d[2]
    t = ((a0 + a1) + a2) / dn
    k = torch.floor((t * 1000.0) / ell)
    h = torch.clamp(k, 1.0, float(HASH_MAX)).to(torch.int64)
    h = torch.where(t >= ell, torch.full_like(h, HASH_MAX), h)
    return torch.where(t > 0.0, h, torch.zeros_like(h))


def _cat(parts):
    return {f: torch.cat([p[f] for p in parts]) for f in parts[0]}


def _take(st, sel):
    return {f: v[sel] for f, v in st.items()}


def _pack(st):
    """Particle records as one FP64 matrix (15 fields, material, label, id) for the collectives."""
    cols = [st[f] for f in STATE] + [st[f].to(torch.float64) for f in INTS]
    return torch.stack(cols, 1) if cols[0].numel() else torch.zeros((0, len(cols)), dtype=torch.float64,
                                                                     device=st["x"].device)


def _unpack(mat):
    st = {f: mat[:, k].contiguous() for k, f in enumerate(STATE)}
    st["mat"] = mat[:, 15].to(torch.uint8)
    st["label"] = mat[:, 16].to(torch.uint8)
    st["id"] = mat[:, 17].to(torch.int64)
    return st


# ------------------------------------------------------------------------------------- collectives
def _allreduce(t, op=dist.ReduceOp.SUM):
    dist.all_reduce(t, op=op)
    return t


def _allgather_rows(mat):
    """All-gather of a variable number of rows (allgatherv): sizes first, then padded blocks."""
    world = dist.get_world_size()
    n = torch.tensor([mat.shape[0]], dtype=torch.int64, device=mat.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n)
    sizes = [int(v.item()) for v in sizes]
    mx = max(sizes)
    pad = torch.zeros((mx, mat.shape[1]), dtype=mat.dtype, device=mat.device)
    pad[: mat.shape[0]] = mat
    blocks = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(blocks, pad)
    return [b[:s] for b, s in zip(blocks, sizes)]


class ShardedSolver:
    """The particles of one label on one rank (rank r owns label r; K = world size)."""

    def __init__(self, scene, engine, device="cpu"):
        self.G = Grid(scene)
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        if self.G.K != self.world:
            raise ValueError("one ownership label per rank: K must equal the world size")
        self.engine = engine
        self.dev = torch.device(device)
        self.swap_period = int(scene.swap_period)
        self.step_index = 0
        mine = np.where(np.asarray(scene.label) == self.rank)[0]
        rho0 = np.array([m[0] for m in scene.materials])[np.asarray(scene.material)]
        v = np.asarray(scene.vel, np.float64)
        st = {"x": scene.pos[:, 0], "y": scene.pos[:, 1], "z": scene.pos[:, 2],
              "vx": v[:, 0], "vy": v[:, 1], "vz": v[:, 2], "w": scene.vol, "m": rho0 * scene.vol,
              "E": 0.5 * ((v[:, 0] * v[:, 0] + v[:, 1] * v[:, 1]) + v[:, 2] * v[:, 2])}
        for f in ("sxx", "syy", "szz", "sxy", "sxz", "syz"):
            st[f] = np.zeros(scene.n)
        self.st = {f: torch.as_tensor(np.ascontiguousarray(st[f][mine]), dtype=torch.float64, device=self.dev)
                   for f in STATE}
        self.st["mat"] = torch.as_tensor(np.asarray(scene.material)[mine], dtype=torch.uint8, device=self.dev)
        self.st["label"] = torch.full((len(mine),), self.rank, dtype=torch.uint8, device=self.dev)
        self.st["id"] = torch.as_tensor(mine, dtype=torch.int64, device=self.dev)
        self.dt = self._global_dt()
        self.last = {}

    # -- time step: the minimum over the ranks of cfl h / max own signal speed (the same FP64 division of
    # the same maximum as on one device)
    def _global_dt(self):
        d = torch.tensor([self.engine.dt(self.st) if self.st["x"].numel() else float("inf")],
                         dtype=torch.float64, device=self.dev)
        return float(_allreduce(d, dist.ReduceOp.MIN).item())

    # -- Sec. III.A / III.B: one swap pass, label pairs in lexicographic order
    def _sums(self, key_types):
        """Fixed-point sums per (label, slot) and counts, summed over the ranks: slot t < nmat for the
        particles of type t, slot nmat for all types."""
        K, T = self.G.K, self.G.nmat + 1
        S = torch.zeros((K, T, 4), dtype=torch.int64, device=self.dev)
        st = self.st
        if st["x"].numel():
            q = [fixed_point(self.G, st[c], a) for a, c in enumerate(("x", "y", "z"))]
            lab = st["label"].to(torch.int64)
            for slot in range(T):
                sel = torch.ones_like(lab, dtype=torch.bool) if slot == self.G.nmat else st["mat"].to(torch.int64) == slot
                for l in torch.unique(lab[sel]).tolist():
                    s2 = sel & (lab == l)
                    for a in range(3):
                        S[l, slot, a] += q[a][s2].sum()
                    S[l, slot, 3] += int(s2.sum())
        return _allreduce(S)

    def _cg(self, S, l, slot):
        cnt = int(S[l, slot, 3])
        if cnt == 0:
            return None
        return [self.G.lo[a] + (float(S[l, slot, a]) / float(cnt)) * self.G.q_step[a] for a in range(3)]

    def swap_pass(self):
        G = self.G
        multi = G.nmat > 1
        moved = 0
        for T in range(G.nmat if multi else 1):
            slot = T if multi else G.nmat
            for a in range(G.K - 1):
                for b in range(a + 1, G.K):
                    S = self._sums(None)
                    ca, cb = self._cg(S, a, slot), self._cg(S, b, slot)
                    if ca is None or cb is None:
                        continue
                    if multi:   # Cg' = alpha Cg_all + (1 - alpha) Cg_type, Cg_all of the same label
                        alla, allb = self._cg(S, a, G.nmat), self._cg(S, b, G.nmat)
                        beta = 1.0 - G.alpha
                        ca = [G.alpha * alla[k] + beta * ca[k] for k in range(3)]
                        cb = [G.alpha * allb[k] + beta * cb[k] for k in range(3)]
                    moved += self._swap_pair(a, b, ca, cb, T if multi else -1)
        return moved

    def _swap_pair(self, a, b, ca, cb, mt):
        st = self.st
        r = self.rank
        h = torch.zeros(st["x"].numel(), dtype=torch.int64, device=self.dev)
        cand = torch.zeros_like(h, dtype=torch.bool)
        if r in (a, b) and st["x"].numel():
            own, oth = (ca, cb) if r == a else (cb, ca)
            M = [(own[k] + oth[k]) * 0.5 for k in range(3)]
            d = [oth[k] - own[k] for k in range(3)]
            dn = float(np.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]))
            if dn > 0.0:
                h = balancing_hash(M, d, dn, dn * 0.5, st["x"], st["y"], st["z"])
                cand = (h > 0) & (st["label"].to(torch.int64) == r)
                if mt >= 0:
                    cand &= st["mat"].to(torch.int64) == mt
        cnt = torch.zeros(2, dtype=torch.int64, device=self.dev)
        if r in (a, b):
            cnt[0 if r == a else 1] = int(cand.sum())
        cnt = _allreduce(cnt)
        m = int(min(cnt[0], cnt[1]))
        if m == 0:
            return 0
        out = None
        if r in (a, b):
            idx = torch.nonzero(cand).flatten()
            # the m highest hashes, ties by the lowest persistent id
            keyv = (HASH_MAX - h[idx]) * (1 << 40) + st["id"][idx]
            pick = idx[torch.argsort(keyv)[:m]]
            keep = torch.ones_like(h, dtype=torch.bool)
            keep[pick] = False
            out = _take(st, pick)
            out["label"] = torch.full((m,), b if r == a else a, dtype=torch.uint8, device=self.dev)
            self.st = _take(st, keep)
        # the two sides exchange their m particles (every rank takes part in the all-gather; the others
        # contribute nothing)
        blocks = _allgather_rows(_pack(out) if out is not None else torch.zeros((0, 18), dtype=torch.float64,
                                                                                device=self.dev))
        if r in (a, b):
            got = _unpack(blocks[b if r == a else a])
            self.st = _cat([self.st, got])
        return 2 * m

    # -- one step in the paper's order
    def step(self):
        G = self.G
        do_swap = self.swap_period > 0 and self.step_index % self.swap_period == 0
        moved = self.swap_pass() if do_swap else 0
        st = self.st
        key = bucket_keys(G, st["x"], st["y"], st["z"])
        # b. hash broadcast as an allreduce (bitwise OR) of the per-bucket label masks
        mask = _allreduce(label_mask(G, key, st["label"].to(torch.int64)), dist.ReduceOp.BOR)
        # c. communication hash and MGPU boundary set
        flag = boundary_flags(G, key, st["label"].to(torch.int64), mask)
        counts = torch.zeros(G.K, dtype=torch.int64, device=self.dev)
        counts[self.rank] = int(flag.sum())
        counts = _allreduce(counts)
        # d. the boundary records into every other rank's halo
        blocks = _allgather_rows(_pack(_take(st, flag)))
        halo = [_unpack(b) for r, b in enumerate(blocks) if r != self.rank and b.shape[0]]
        union = _cat([st] + halo) if halo else st
        # e-g. interaction of the own particles with own and halo particles, integration of the own
        new, nreal, nimage = self.engine.advance(union, st["x"].numel(), self.dt)
        self.last = {"key": key, "flag": flag, "comm": torch.where(flag, key, torch.full_like(key, G.ncell)),
                     "id": st["id"].clone(), "counts": counts, "moved": moved, "halo": int(union["x"].numel() - st["x"].numel()),
                     "nreal": nreal, "nimage": nimage, "dt": self.dt}
        self.st = new
        self.dt = self._global_dt()
        self.step_index += 1

    def gather(self):
        """The whole particle set on every rank (ids and fields as numpy arrays, sorted by id)."""
        parts = [None] * self.world
        dist.all_gather_object(parts, {f: v.cpu().numpy() for f, v in self.st.items()})
        allp = {f: np.concatenate([p[f] for p in parts]) for f in parts[0]}
        o = np.argsort(allp["id"])
        return {f: v[o] for f, v in allp.items()}


class GpuEngine:
    """Interaction and integration on this rank's GPU through libgsph (FP64 or FP32-split): a context of
    the rank's own and halo particles takes one step with the given time step (one label, no swap pass),
    and the own particles' new state is kept; the time step of the own particles comes from a context of
    those alone."""

    def __init__(self, scene, precision: int, device: int = 0):
        import copy

        from . import gsph
        self.gsph = gsph
        sc = copy.deepcopy(scene)
        sc.K, sc.swap_period = 1, 0
        self.cfg = gsph.config_from_scene(sc, precision=precision, device=device, diagnostics=True)
        self.device = device

    def _ctx(self, st):
        n = st["x"].numel()
        sol = self.gsph.Solver(self.cfg)
        pos = torch.stack([st["x"], st["y"], st["z"]], 1).contiguous()
        vel = torch.stack([st["vx"], st["vy"], st["vz"]], 1).contiguous()
        sol.set_particles(pos, vel, st["w"].contiguous(), st["mat"].contiguous(),
                          torch.zeros(n, dtype=torch.uint8, device=pos.device))
        for f in STATE:
            sol.put(f, st[f].contiguous())
        sol.put("id", torch.arange(n, dtype=torch.int32, device=pos.device))
        return sol

    def advance(self, union, n_own: int, dt: float):
        sol = self._ctx(union)
        sol.set_dt(dt)
        sol.step(1)
        sol.sync()
        slot = torch.empty(union["x"].numel(), dtype=torch.int32, device=union["x"].device)
        sol.get_into("id", slot)
        own = slot < n_own   # the library's ids are the input order: the own particles come first
        new = {}
        for f in STATE:
            t = torch.empty_like(union[f])
            sol.get_into(f, t)
            new[f] = t[own]
        src = slot[own].to(torch.int64)
        for f in INTS:
            new[f] = union[f][src]
        nr = torch.empty(union["x"].numel(), dtype=torch.int32, device=union["x"].device)
        ni = torch.empty_like(nr)
        sol.get_into("nreal", nr)
        sol.get_into("nimage", ni)
        sol.close()
        return new, nr[own], ni[own]

    def dt(self, st):
        sol = self._ctx(st)
        v = sol.dt()
        sol.close()
        return v
