"""Differentiable distortion of a codebook: a torch.autograd.Function over the C ABI.

    D = sum_m min_n ||x_m - c_n||^2            (Sec. 2.2 distortion, summed)

The forward pass is the library's nearest-codevector search (vq_encode); the
backward pass differentiates D at the fixed cell table found by the forward
pass (lbg_distortion_backward):

    dD/dc_n = 2 (count_n c_n - sum_{a(m)=n} x_m),   dD/dx_m = 2 (x_m - c_a(m)).

These are the true gradients wherever no vector sits on a tie between two
codevectors (where D is not differentiable).  Both kernels run on the GPU;
this module only marshals tensors.  For CUDA tensors neither pass waits for
the device: D is a device scalar written by the forward call, and the
upstream gradient is handed to the backward kernels as a device scalar.
"""
from __future__ import annotations

import torch

from . import _binding


class Distortion(torch.autograd.Function):
    """D(X, C) with the nearest-codevector cell table (see the module docstring)."""

    @staticmethod
    def forward(ctx, X: torch.Tensor, C: torch.Tensor, precision: str = "fp32"):
        X = X.detach().contiguous()
        C = C.detach().contiguous()
        if X.is_cuda and C.is_cuda:
            buf = _binding.step_result_buffer(X.device)
            enc = _binding.vq_encode(X, C, precision=precision, result_out=buf)
            D = buf[:8].view(torch.float64).reshape(())       # written on the device
        else:
            enc = _binding.vq_encode(X, C, precision=precision)
            D = torch.tensor(enc.D, dtype=torch.float64, device=X.device)
        ctx.save_for_backward(X, C, enc.idx)
        return D

    @staticmethod
    def backward(ctx, grad_D):
        X, C, idx = ctx.saved_tensors
        need_x, need_c = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if X.is_cuda:
            g = grad_D.detach().to(device=X.device, dtype=torch.float32).reshape(1).contiguous()
            buf = _binding.step_result_buffer(X.device)
            _, dC, dX, _ = _binding.distortion_backward(X, C, idx, want_dC=need_c, want_dX=need_x,
                                                        grad_scale=g, result_out=buf)
        else:
            _, dC, dX, _ = _binding.distortion_backward(X, C, idx, float(grad_D), want_dC=need_c,
                                                        want_dX=need_x)
        return dX, dC, None


def distortion(X: torch.Tensor, C: torch.Tensor, precision: str = "fp32") -> torch.Tensor:
    """Differentiable total distortion of X under codebook C (0-dim float64 tensor)."""
    return Distortion.apply(X, C, precision)
