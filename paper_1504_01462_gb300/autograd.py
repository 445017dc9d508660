"""torch.autograd.Function over pw_grad: the weighted summed transmission
sum_i w_i T(E_i, k_par_i) as a differentiable function of the device wells'
depths V0 and of one geometry parameter (the sheet gap of a side-contact
junction).

The forward pass builds a context for the given parameters and runs the FP64
adjoint (pw_grad), which returns the sum together with its derivatives; the
backward pass only scales them by the incoming gradient.  Torch is used for the
autograd bookkeeping only: every number comes from the CUDA path."""
from __future__ import annotations

import numpy as np
import torch

from . import Context  # noqa: F401  (the contexts the factory returns)


class SummedTransmission(torch.autograd.Function):
    """apply(v0, gap, make_context, E, kpar, weight) -> sum_i w_i T_i.

    v0            1-D float64 tensor of the device wells' depths (Ry)
    gap           0-d float64 tensor (the geometry parameter, in the unit the
                  factory takes)
    make_context  callable (v0 ndarray, gap float) -> Context whose setup
                  carries the wells' and electrodes' motion per unit gap
    E, kpar       host arrays of the points; weight: host array or None
    """

    @staticmethod
    def forward(ctx, v0, gap, make_context, E, kpar, weight):
        with make_context(v0.detach().cpu().numpy().astype(np.float64), float(gap)) as pc:
            sumT, dV0, dgap = pc.grad(E, kpar, weight, n_wells=v0.numel(), gap=True)
        ctx.save_for_backward(torch.as_tensor(dV0, dtype=torch.float64),
                              torch.tensor(dgap, dtype=torch.float64))
        return torch.tensor(sumT, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        dV0, dgap = ctx.saved_tensors
        return grad_out * dV0, grad_out * dgap, None, None, None, None


def summed_transmission(v0, gap, make_context, E, kpar, weight=None):
    return SummedTransmission.apply(v0, gap, make_context, E, kpar, weight)


__all__ = ["SummedTransmission", "summed_transmission"]
