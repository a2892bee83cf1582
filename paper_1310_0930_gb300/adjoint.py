"""Differentiable LWFA objective: a ``torch.autograd.Function`` whose forward
runs the GB300 timestep (with checkpoints) and whose backward runs the
library's hand-written adjoint kernels (reverse sweep with segment
recomputation).  Inputs: the density-profile knots and the laser amplitude
a0; output: the weighted mean kinetic energy of the electrons inside a
smooth window of the last axis at the final step."""
from __future__ import annotations

import copy
import dataclasses

import numpy as np
import torch

from . import inputs
from .sim import Simulation


@dataclasses.dataclass
class Objective:
    z_lo: float    # window-frame cells along the last axis
    z_hi: float
    width: float = 1.0


def _workload(base: inputs.Workload, knots: np.ndarray, a0: float) -> inputs.Workload:
    w = copy.deepcopy(base)
    w.knots = np.asarray(knots, dtype=np.float64)
    if w.knot_z == (0.0, 0.0):
        w.knot_z = (0.0, w.n[-1] * w.d[-1])
    w.laser.a0 = float(a0)
    return w


class LWFAObjective(torch.autograd.Function):
    """L(knots, a0) = sum w K sigma / sum w sigma after `steps` steps."""

    @staticmethod
    def forward(ctx, knots: torch.Tensor, a0: torch.Tensor, base: inputs.Workload, obj: Objective,
                steps: int, checkpoint_every: int):
        w = _workload(base, knots.detach().cpu().numpy(), float(a0.detach().cpu()))
        parts = inputs.background(w)
        sim = Simulation(w, track_ids=True, per_particle_weight=True)
        sim.load(parts)
        sim.adjoint_begin(steps, checkpoint_every)
        sim.step(steps)
        L = sim.objective(obj.z_lo, obj.z_hi, obj.width)
        ctx.sim, ctx.obj, ctx.n_knots = sim, obj, int(knots.numel())
        ctx.dtype, ctx.device = knots.dtype, knots.device
        return torch.tensor(L, dtype=knots.dtype, device=knots.device)

    @staticmethod
    def backward(ctx, g):
        sim, obj = ctx.sim, ctx.obj
        res = sim.adjoint_backward(obj.z_lo, obj.z_hi, obj.width, n_knots=ctx.n_knots)
        sim.close()
        gk = torch.tensor(res["dL_dknots"], dtype=ctx.dtype, device=ctx.device) * g
        ga = torch.tensor(res["dL_da0"], dtype=ctx.dtype, device=ctx.device) * g
        return gk, ga, None, None, None, None


def objective(knots: torch.Tensor, a0: torch.Tensor, base: inputs.Workload, obj: Objective, steps: int,
              checkpoint_every: int = 100) -> torch.Tensor:
    return LWFAObjective.apply(knots, a0, base, obj, steps, checkpoint_every)
