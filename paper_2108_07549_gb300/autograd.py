"""torch.autograd binding of the differentiated form (pdr_backward).

``unrolled_objective(solver, u, d, T, ckpt_every)`` returns the tensor
L(u, d) = z(f^(T)): the objective of Alg. 1 (arXiv 2108.07549) after T sweeps
from f = 0 on the instance held by ``solver`` with capacities u and demands d.
Its backward pass is the library's reverse mode through the T sweeps
(hand-written CUDA kernels, checkpointed every ``ckpt_every`` sweeps), so
``L.backward()`` fills ``u.grad`` and ``d.grad``: the sensitivity of the
remaining infeasibility to each capacity (for capacity upgrades) and each
demand.  The forward pass runs only the T sweeps; the backward pass re-runs
them with checkpoints.
"""

from __future__ import annotations

import numpy as np
import torch


class _UnrolledObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, d, solver, T, ckpt_every):
        solver.set_data(u.detach().cpu().double().numpy(), d.detach().cpu().double().numpy())
        L, _, _ = solver.backward(int(T), int(ckpt_every), grads=False)
        ctx.solver, ctx.T, ctx.ckpt = solver, int(T), int(ckpt_every)
        ctx.u_np = u.detach().cpu().double().numpy()
        ctx.d_np = d.detach().cpu().double().numpy()
        ctx.dtype_u, ctx.dev_u, ctx.dtype_d, ctx.dev_d = u.dtype, u.device, d.dtype, d.device
        return torch.tensor(L, dtype=u.dtype, device=u.device)

    @staticmethod
    def backward(ctx, grad_out):
        solver = ctx.solver
        solver.set_data(ctx.u_np, ctx.d_np)
        _, gu, gd = solver.backward(ctx.T, ctx.ckpt, grads=True)
        g = float(grad_out.detach().cpu())
        gu_t = torch.from_numpy(np.asarray(gu) * g).to(device=ctx.dev_u, dtype=ctx.dtype_u)
        gd_t = torch.from_numpy(np.asarray(gd) * g).to(device=ctx.dev_d, dtype=ctx.dtype_d)
        return gu_t, gd_t, None, None, None


def unrolled_objective(solver, u: torch.Tensor, d: torch.Tensor, T: int, ckpt_every: int = 10) -> torch.Tensor:
    """L(u, d) = z(f^(T)) as a differentiable torch scalar (see the module docstring)."""
    return _UnrolledObjective.apply(u, d, solver, T, ckpt_every)
