"""torch.autograd binding of the differentiated form (pdr_backward).

``unrolled_objective(solver, u, d, T, ckpt_every)`` returns the tensor
L(u, d) = z(f^(T)): the objective of Alg. 1 (arXiv 2108.07549) after T sweeps
from f = 0 on the instance held by ``solver`` with capacities u and demands d.
Its backward pass is the library's reverse mode through the T sweeps
(hand-written CUDA kernels, checkpointed every ``ckpt_every`` sweeps), so
``L.backward()`` fills ``u.grad`` and ``d.grad``: the sensitivity of the
remaining infeasibility to each capacity (for capacity upgrades) and each
demand.

CUDA tensors stay on the device: u and d reach the library as device
pointers (pdr_set_data checks and converts them there) and the gradients are
written by pdr_backward into device tensors.  When a gradient is wanted the
forward pass runs the reverse mode at once (one pass of T sweeps forward and
the checkpointed backward), and the backward pass only scales the stored
gradients by the incoming one.  CPU tensors go through host memory.
"""

from __future__ import annotations

import torch


def _as_f64(x: torch.Tensor) -> torch.Tensor:
    return x.detach().to(dtype=torch.float64).contiguous()


class _UnrolledObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u, d, solver, T, ckpt_every):
        want = ctx.needs_input_grad[0] or ctx.needs_input_grad[1]
        u64, d64 = _as_f64(u), _as_f64(d)
        if u64.is_cuda and d64.is_cuda:
            # the library runs on its own stream: the converted inputs must be ready
            torch.cuda.current_stream(u64.device).synchronize()
            solver.set_data_device(u64.data_ptr(), d64.data_ptr())
            gu = torch.empty_like(u64) if want else None
            gd = torch.empty_like(d64) if want else None
            L = solver.backward_into(int(T), int(ckpt_every), gu.data_ptr() if want else 0,
                                     gd.data_ptr() if want else 0)
        else:
            solver.set_data(u64.cpu().numpy(), d64.cpu().numpy())
            L, gu_np, gd_np = solver.backward(int(T), int(ckpt_every), grads=want)
            gu = torch.from_numpy(gu_np) if want else None
            gd = torch.from_numpy(gd_np) if want else None
        if want:
            ctx.save_for_backward(gu.to(u.device), gd.to(d.device))
        ctx.dtypes = (u.dtype, d.dtype)
        return torch.tensor(L, dtype=u.dtype, device=u.device)

    @staticmethod
    def backward(ctx, grad_out):
        gu, gd = ctx.saved_tensors
        g = grad_out.to(torch.float64)
        return (gu * g).to(ctx.dtypes[0]), (gd * g).to(ctx.dtypes[1]), None, None, None


def unrolled_objective(solver, u: torch.Tensor, d: torch.Tensor, T: int, ckpt_every: int = 10) -> torch.Tensor:
    """L(u, d) = z(f^(T)) as a differentiable torch scalar (see the module docstring)."""
    return _UnrolledObjective.apply(u, d, solver, T, ckpt_every)
