"""The energy as a differentiable function of the positions (torch.autograd).

The forward pass is one evaluation by the library (energy, forces, virial
and per-atom energies on the device, Sec. 2.1); the backward pass returns
-F times the incoming gradient, since the kernels compute the forces as the
exact negative gradient of the energy they compute, so no second evaluation
runs.  The virial (-dE/d strain for a homogeneous strain of box and
positions) and the per-atom energies are returned as non-differentiable
outputs; gradients with respect to the model parameters are not provided.
"""
from __future__ import annotations

import torch

from . import dp


class _Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, types, box, handle):
        E, F, V, Ei = dp.dp_compute(handle, x.detach().contiguous(), types, box, atom_energy=True)
        ctx.save_for_backward(F)
        ctx.mark_non_differentiable(V, Ei)
        return E[0], V, Ei

    @staticmethod
    def backward(ctx, gE, gV, gEi):
        (F,) = ctx.saved_tensors
        gx = None
        if ctx.needs_input_grad[0]:
            gx = -gE * F
        return gx, None, None, None


def energy(handle, x: torch.Tensor, types: torch.Tensor, box: torch.Tensor):
    """E (0-dim FP64 tensor, differentiable in x), virial [3, 3], per-atom
    energies [N].  x: CUDA FP64 [N, 3] (A); types: CUDA int32 [N]; box: CUDA
    FP64 [3, 3] (orthorhombic)."""
    if not (x.is_cuda and x.dtype == torch.float64 and x.dim() == 2 and x.shape[1] == 3):
        raise ValueError("x must be a CUDA float64 tensor of shape [N, 3]")
    return _Energy.apply(x, types, box, handle)
