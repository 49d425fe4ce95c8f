"""torch.autograd.Function over the adjoint-gradient path.

``energy(thetas, gates, hamiltonian, n)`` returns E(theta) for a batch of
parameter sets ``thetas`` [B, P] (float64 tensor; P = number of RX/RY/RZ
gates without controls, in circuit order).  The forward call runs the CUDA
adjoint sweep, which yields the energies and all gradients in one pass; the
backward call only scales the stored gradients by the incoming grad_output.
"""
from __future__ import annotations

import numpy as np
import torch

from . import qcgb300 as q


class AdjointEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, thetas, gates, hamiltonian, n, dtype, arith):
        th = thetas.detach().to("cpu", torch.float64).numpy()
        e, g = q.adjoint_grad(n, gates, hamiltonian, th, dtype=dtype, arith=arith)
        ctx.save_for_backward(torch.from_numpy(np.ascontiguousarray(g)).to(thetas.device, thetas.dtype))
        return torch.from_numpy(e).to(thetas.device, thetas.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out[:, None] * g, None, None, None, None, None


def energy(thetas: torch.Tensor, gates, hamiltonian, n: int, dtype: int = q.C64, arith: int = q.ARITH_AUTO):
    """Batched energies E(theta) [B] with adjoint gradients for autograd."""
    if thetas.dim() == 1:
        return AdjointEnergy.apply(thetas[None, :], gates, hamiltonian, n, dtype, arith)[0]
    return AdjointEnergy.apply(thetas, gates, hamiltonian, n, dtype, arith)
