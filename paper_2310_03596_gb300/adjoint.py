"""Gradient of an impact observable through the library's checkpointed adjoint (gsph_adjoint).

Observable J = mean z velocity, after N steps, of the rear-face particles: those whose initial lattice
z index is the top layer of the impacting cube. Parameters theta = (Y, G, v0): yield stress and shear
modulus of material 0, and the initial z velocity of every particle.

Everything runs inside the library: the forward in the context's precision with a device checkpoint
every `every` steps, the recompute of each segment from its checkpoint, the FP64 reverse steps, and the
assembly of dJ/dY, dJ/dG and dJ/dv0. The time-step schedule is part of J's definition: given, or the
forward's own CFL steps, which the gradient then holds fixed. This module only builds the scene for a
parameter vector and wraps the call in a torch.autograd.Function.
"""
from __future__ import annotations

import copy

import numpy as np

from . import gsph


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


def observable(scene, steps: int, every: int, precision: int, dts=None, want_gradient: bool = True,
               device: int = 0):
    """(J, (dJ/dY, dJ/dG, dJ/dv0) or None, schedule) of the scene by one gsph_adjoint call."""
    sol = gsph.Solver.from_scene(scene, precision=precision, device=device)
    try:
        return sol.adjoint(steps, every, rear_face_ids(scene), dts=dts, want_gradient=want_gradient)
    finally:
        sol.close()


def impact_observable(scene, theta, steps: int = 200, every: int = 20, precision: int = gsph.FP32_SPLIT,
                      dts=None):
    """J(theta) as a torch scalar differentiable w.r.t. theta = tensor([Y, G, v0]) (float64, CPU). J is
    defined on the time-step schedule dts (steps values), or, when dts is None, on the schedule of the
    forward run at theta, held fixed; the gradient is that of this J."""
    import torch

    class _ImpactObservable(torch.autograd.Function):
        @staticmethod
        def forward(ctx, th):
            Y, G, v0 = (float(v) for v in th.detach().cpu())
            J, g, _ = observable(with_parameters(scene, Y, G, v0), steps, every, precision, dts=dts)
            ctx.g = g
            return torch.tensor(J, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gJ):
            return gJ * torch.tensor(ctx.g, dtype=torch.float64)

    return _ImpactObservable.apply(theta)
