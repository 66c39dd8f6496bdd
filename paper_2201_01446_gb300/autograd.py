"""The energy as a differentiable function of the positions (torch.autograd).

The forward pass is one evaluation by the library (energy, forces, virial
and per-atom energies on the device, Sec. 2.1); the backward pass returns
-F times the incoming gradient, since the kernels compute the forces as the
exact negative gradient of the energy they compute, so no second evaluation
runs.  The virial (-dE/d strain for a homogeneous strain of box and
positions) and the per-atom energies are returned as non-differentiable
outputs.

energy_params is the energy as a function of the model's parameters (the
fitting nets' weights and biases and the table coefficients, in the flat
layouts of dp_param_grad): its forward loads the given values into the
handle and runs one evaluation that also returns dE/d(parameters), which
the backward scales by the incoming gradient.
"""
from __future__ import annotations

import numpy as np
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


class _EnergyParams(torch.autograd.Function):
    @staticmethod
    def forward(ctx, fit, table, handle, x, types, box):
        dp.dp_set_params(handle, fit.detach().cpu().numpy(),
                         table.detach().cpu().numpy() if table is not None else None)
        E, gf, gt = dp.dp_param_grad(handle, x, types, box, table=table is not None)
        ctx.save_for_backward(torch.from_numpy(gf),
                              torch.from_numpy(gt) if gt is not None else torch.zeros(0))
        ctx.has_table = table is not None
        return torch.tensor(E, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gE):
        gf, gt = ctx.saved_tensors
        return gE * gf, (gE * gt if ctx.has_table else None), None, None, None, None


def _host(a, dtype):
    if isinstance(a, torch.Tensor):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype)


def energy_params(handle, fit: torch.Tensor, table, x, types, box):
    """E (0-dim FP64 CPU tensor) as a differentiable function of the fitting
    parameters fit [n_fit] and the embedding representation table [n_table]
    or None (the table coefficients of a tabulated tensor-core handle, the
    embedding nets' weights and biases of an untabulated one); both CPU
    float64 tensors in the layouts of dp_param_grad.  x [N, 3], types [N],
    box [3, 3]: host arrays or tensors (copied to the host).  The handle
    keeps the given parameters afterwards."""
    if fit.dtype != torch.float64 or (table is not None and table.dtype != torch.float64):
        raise ValueError("parameters must be float64 tensors")
    return _EnergyParams.apply(fit, table, handle, _host(x, np.float64), _host(types, np.int32),
                               _host(box, np.float64))
