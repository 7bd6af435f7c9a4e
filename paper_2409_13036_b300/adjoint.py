"""torch.autograd bridge of the differentiation form (rafem_tape_begin / rafem_adjoint).

`final_temperature(model, sigma0, k, n_steps)` runs n_steps lagged time steps of a library context from its
initial condition (or a given initial temperature) with the per-element conductivities taken from the tensors
sigma0 and k, and returns the final temperature field as a differentiable FP64 CUDA tensor. Its backward pass is
the library's discrete adjoint: transposed (here: symmetric) solves of the thermal and potential systems, step by
step back to the start, with the forward states recomputed from checkpoints every `checkpoint_every` steps.
Parameters may be FP32 (the usual storage of trainable tensors); they are widened to FP64 on the device before
the library reads them, and the gradients come back in the parameters' dtype.

Argument marshalling only: every arithmetic step of the forward and backward passes runs in librafem's kernels.
The library works on its own CUDA stream; the wrapper synchronises torch's current stream before each call (the
library synchronises its stream before returning).
"""
from __future__ import annotations

import torch

from . import rafem


def _sync():
    torch.cuda.current_stream().synchronize()


class RafemFinalTemperature(torch.autograd.Function):
    """T^N = F(sigma0, k, T0); see the module docstring."""

    @staticmethod
    def forward(ctx, sigma0, k, T0, model, n_steps, checkpoint_every):
        dev = sigma0.device
        s64 = sigma0.detach().to(torch.float64).contiguous()
        k64 = k.detach().to(torch.float64).contiguous()
        _sync()
        model.set_params(s64, k64)
        model.reset()
        if T0 is not None:
            t0 = T0.detach().to(torch.float64).contiguous()
            _sync()
            model.set_state_device(T=t0, step=0)
        model.tape_begin(checkpoint_every)
        status, st = model.run(n_steps)
        ctx.forward_stats = st.as_dict()
        T = torch.empty(model.N, dtype=torch.float64, device=dev)
        model.get_field_device(rafem.RAFEM_SYS_T, T)
        ctx.model = model
        ctx.dtypes = (sigma0.dtype, k.dtype, None if T0 is None else T0.dtype)
        return T

    @staticmethod
    def backward(ctx, grad_T):
        model = ctx.model
        dev = grad_T.device
        gT = grad_T.detach().to(torch.float64).contiguous()
        gs = torch.empty(model.n_tets, dtype=torch.float64, device=dev)
        gk = torch.empty(model.n_tets, dtype=torch.float64, device=dev)
        g0 = torch.empty(model.N, dtype=torch.float64, device=dev)
        _sync()
        _, st = model.adjoint_ptr(gT, None, 1, gs, gk, g0, 1)
        ctx.adjoint_stats = st
        ds, dk, dt0 = ctx.dtypes
        return gs.to(ds), gk.to(dk), (None if dt0 is None else g0.to(dt0)), None, None, None


def final_temperature(model: "rafem.Context", sigma0: torch.Tensor, k: torch.Tensor, n_steps: int,
                      checkpoint_every: int = 10, T0: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable final temperature of `model` after n_steps steps (sigma0, k: CUDA tensors [E] in mesh
    element order; T0: optional CUDA tensor [N])."""
    return RafemFinalTemperature.apply(sigma0, k, T0, model, int(n_steps), int(checkpoint_every))
