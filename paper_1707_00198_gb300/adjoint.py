"""torch.autograd.Function around the hand-written adjoint of the step (lbcg_adjoint).

``WettingObjective.apply(theta_node, sigma, nu_R, nu_B, spec)`` runs the colour-gradient LBM
with the improved wetting condition (Sec. II) from the geometry's initial state for
``spec.nsteps`` steps on the GPU and returns the objective J at the last step (finger length
x_tip - x_cl of Sec. III.D, the red mass, or a weighted sum of rho^N).  Its backward gives
dJ/d(theta per node), dJ/d sigma, dJ/d nu_R and dJ/d nu_B from the same call: the reverse
sweep runs in the forward of this Function and its results are kept for backward.  Any
further dependence (the viscosity ratio M = nu_R / nu_B, a global angle broadcast to the
wall nodes) follows by torch's chain rule.  One lattice per call; the forward runs in the
spec's precision (FP64, or FP32 with an FP64 reverse sweep).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import torch

from .inputs import Geometry, Params
from .lbcg import Lattice


@dataclasses.dataclass
class ObjectiveSpec:
    geom: Geometry
    params: Params
    nsteps: int
    checkpoint: int
    objective: str = "finger_length"       # "finger_length", "red_mass" or "weighted"
    weight: Optional[np.ndarray] = None    # [ny, nx], for "weighted"
    precision: str = "fp64"                # "fp64" or "fp32" (forward steps and checkpoints)
    reverse: str = "fp64"                  # "fp64" or "fp32" (arithmetic of the reverse sweep)


class WettingObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta_node, sigma, nu_R, nu_B, spec: ObjectiveSpec):
        th = theta_node.detach().to("cpu", torch.float64).numpy()
        g = dataclasses.replace(spec.geom, theta_node=np.ascontiguousarray(th))
        p = dataclasses.replace(spec.params, sigma=float(sigma), nu_R=float(nu_R), nu_B=float(nu_B),
                                theta=float(th.mean()))
        L = Lattice(g, p, spec.precision)
        try:
            rev = spec.reverse == "fp32"
            if spec.objective == "weighted":
                out = L.adjoint(spec.nsteps, spec.checkpoint, weight=spec.weight, reverse_fp32=rev)
            else:
                out = L.adjoint(spec.nsteps, spec.checkpoint, objective=spec.objective, reverse_fp32=rev)
        finally:
            L.close()
        f64 = dict(dtype=torch.float64)
        ctx.save_for_backward(torch.as_tensor(out["dtheta_node"], **f64), torch.tensor(out["dsigma"], **f64),
                              torch.tensor(out["dnu_R"], **f64), torch.tensor(out["dnu_B"], **f64))
        ctx.devices = (theta_node.device, getattr(sigma, "device", None))
        return torch.tensor(out["J"], **f64)

    @staticmethod
    def backward(ctx, gJ):
        dth, ds, dR, dB = ctx.saved_tensors
        gJ = gJ.to(torch.float64).cpu()
        return (gJ * dth).to(ctx.devices[0]), gJ * ds, gJ * dR, gJ * dB, None


def objective(theta_node: torch.Tensor, sigma: torch.Tensor, nu_R: torch.Tensor, nu_B: torch.Tensor,
              spec: ObjectiveSpec) -> torch.Tensor:
    """J at step spec.nsteps as a differentiable function of the wetting and fluid parameters."""
    return WettingObjective.apply(theta_node, sigma, nu_R, nu_B, spec)
