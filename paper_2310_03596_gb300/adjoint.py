"""Gradient of an impact observable through the hand-written adjoint of the step.

Observable J = mean z velocity, after N steps, of the rear-face particles: those whose initial lattice
z index is the top layer of the impacting cube. Parameters theta = (Y, G, v0): yield stress and shear
modulus of material 0, and the initial z velocity of every particle.

Forward: the configured precision, a device checkpoint of the full state every `every` steps, and the
dt of every step recorded. Backward: for each segment in reverse, the segment's states are recomputed
from its checkpoint with the recorded dts (bit for bit, the kernels are deterministic), then
gsph_adjoint_step (reverse mode of interaction + integration, FP64, neighbour set and dt of the step
held fixed) runs backwards through the segment. Memory: the checkpoints plus one segment of states.

The gradient w.r.t. v0 comes from the adjoint of the initial state: v_z of every particle equals v0
and the specific total energy E = |v|^2 / 2 carries dE/dv0 = v_z.
"""
from __future__ import annotations

import copy

import numpy as np

from . import gsph

STATE_FIELDS = tuple(gsph.FIELDS[:15])
INT_FIELDS = ("material", "label", "id")
FVZ, FE = STATE_FIELDS.index("vz"), STATE_FIELDS.index("E")


def with_parameters(scene, Y: float, G: float, v0: float):
    """A copy of the scene with material 0's yield stress and shear modulus and the initial z
    velocity replaced."""
    s = copy.deepcopy(scene)
    mats = list(s.materials)
    rho0, K, _, _ = mats[0]
    mats[0] = (rho0, K, G, Y)
    s.materials = mats
    s.vel = s.vel.copy()
    s.vel[:, 2] = v0
    return s


def rear_face_ids(scene) -> np.ndarray:
    """Persistent ids of the particles on the top lattice layer (the rear face of a cube moving
    towards -z)."""
    layer = np.rint(scene.pos[:, 2] / scene.dx - 0.5).astype(np.int64)
    return np.where(layer == layer.max())[0].astype(np.uint32)


def _snapshot(sol, stream=None):
    import torch
    snap = {}
    for f in STATE_FIELDS:
        t = torch.empty(sol.n, dtype=torch.float64, device="cuda")
        sol.get_into(f, t, stream)
        snap[f] = t
    for f, dt in (("material", torch.uint8), ("label", torch.uint8), ("id", torch.int32)):
        t = torch.empty(sol.n, dtype=dt, device="cuda")
        sol.get_into(f, t, stream)
        snap[f] = t
    return snap


def _restore(sol, snap, stream=None):
    for f in STATE_FIELDS + INT_FIELDS:
        sol.put(f, snap[f], stream)


class ForwardRecord:
    """A forward run with checkpoints, ready for the reverse sweep."""

    def __init__(self, scene, steps: int, every: int, precision: int, device: int = 0):
        import torch

        self.scene, self.steps, self.every, self.precision = scene, steps, every, precision
        self.fwd = gsph.Solver.from_scene(scene, precision=precision, device=device)
        self.dts = []
        self.ckpts = {}
        for k in range(steps):
            if k % every == 0:
                self.ckpts[k] = _snapshot(self.fwd)
            self.dts.append(self.fwd.dt())
            self.fwd.step(1)
        self.fwd.sync()
        rear = rear_face_ids(scene)
        ids = self.fwd.get("id")
        mask = np.isin(ids, rear)
        vz = self.fwd.get("vz")
        self.J = float(vz[mask].mean())
        self.lam_final = torch.zeros((15, scene.n), dtype=torch.float64, device="cuda")
        self.lam_final[FVZ][torch.from_numpy(mask).cuda()] = 1.0 / mask.sum()

    def gradient(self, device: int = 0):
        """(dJ/dY, dJ/dG, dJ/dv0) by the reverse sweep."""
        import torch

        adj = gsph.Solver.from_scene(self.scene, precision=gsph.FP64, device=device, diagnostics=True)
        lam = self.lam_final.clone()
        lam_prev = torch.empty_like(lam)
        gY = gG = 0.0
        starts = sorted(self.ckpts)
        for si in reversed(range(len(starts))):
            k0 = starts[si]
            k1 = starts[si + 1] if si + 1 < len(starts) else self.steps
            _restore(self.fwd, self.ckpts[k0])
            states = [self.ckpts[k0]]
            for k in range(k0, k1 - 1):
                self.fwd.set_dt(self.dts[k])
                self.fwd.step(1)
                states.append(_snapshot(self.fwd))
            for k in reversed(range(k0, k1)):
                _restore(adj, states[k - k0])
                y, g = adj.adjoint_step(lam, lam_prev, self.dts[k])
                gY += y
                gG += g
                lam, lam_prev = lam_prev, lam
        torch.cuda.synchronize()
        vz0 = torch.from_numpy(np.ascontiguousarray(self.scene.vel[:, 2])).cuda()
        g_v0 = float(lam[FVZ].sum() + (lam[FE] * vz0).sum())
        adj.close()
        return gY, gG, g_v0

    def close(self):
        self.fwd.close()


def impact_observable(scene, theta, steps: int = 200, every: int = 20, precision: int = gsph.FP32_SPLIT):
    """J(theta) as a torch scalar differentiable w.r.t. theta = tensor([Y, G, v0]) (float64, CPU)."""
    import torch

    class _ImpactObservable(torch.autograd.Function):
        @staticmethod
        def forward(ctx, th):
            Y, G, v0 = (float(v) for v in th.detach().cpu())
            rec = ForwardRecord(with_parameters(scene, Y, G, v0), steps, every, precision)
            ctx.rec = rec
            return torch.tensor(rec.J, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gJ):
            g = ctx.rec.gradient()
            ctx.rec.close()
            return gJ * torch.tensor(g, dtype=torch.float64)

    return _ImpactObservable.apply(theta)
