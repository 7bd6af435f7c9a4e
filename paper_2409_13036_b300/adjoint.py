"""torch.autograd bridge of the differentiation form (rafem_tape_begin / rafem_adjoint).

`final_temperature(model, sigma0, k, n_steps)` runs n_steps lagged time steps of a library context from its
initial condition (or a given initial temperature) with the per-element conductivities taken from the tensors
sigma0 and k, and returns the final temperature field as a differentiable FP64 CUDA tensor. Its backward pass is
the library's discrete adjoint: transposed (here: symmetric) solves of the thermal and potential systems, step by
step back to the start, with the forward states recomputed from checkpoints every `checkpoint_every` steps.
Parameters may be FP32 (the usual storage of trainable tensors: passed to rafem_set_params_device, which widens
them to FP64 in the library) or FP64 (rafem_set_params), both of one dtype; the gradients come back in that dtype
(rafem_adjoint writes FP32 gradients itself when the parameters are FP32). The initial temperature, when given,
is an FP64 tensor.

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
        if sigma0.dtype != k.dtype or sigma0.dtype not in (torch.float32, torch.float64):
            raise TypeError("sigma0 and k must both be float32 or both float64 tensors")
        if T0 is not None and T0.dtype != torch.float64:
            raise TypeError("T0 must be a float64 tensor")
        s = sigma0.detach().contiguous()
        kk = k.detach().contiguous()
        _sync()
        if s.dtype == torch.float32:
            model.set_params_device(s, kk)
        else:
            model.set_params(s, kk)
        model.reset()
        if T0 is not None:
            t0 = T0.detach().contiguous()
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
        gT = grad_T.detach().contiguous()  # FP64, the dtype of the forward's output
        ds, _, dt0 = ctx.dtypes
        gs = torch.empty(model.n_tets, dtype=ds, device=dev)
        gk = torch.empty(model.n_tets, dtype=ds, device=dev)
        g0 = torch.empty(model.N, dtype=torch.float64, device=dev)
        _sync()
        _, st = model.adjoint_ptr(gT, None, 1, gs, gk, g0, 2 if ds == torch.float32 else 1)
        ctx.adjoint_stats = st
        return gs, gk, (None if dt0 is None else g0), None, None, None


def final_temperature(model: "rafem.Context", sigma0: torch.Tensor, k: torch.Tensor, n_steps: int,
                      checkpoint_every: int = 10, T0: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable final temperature of `model` after n_steps steps (sigma0, k: CUDA tensors [E] in mesh
    element order; T0: optional CUDA tensor [N])."""
    return RafemFinalTemperature.apply(sigma0, k, T0, model, int(n_steps), int(checkpoint_every))
