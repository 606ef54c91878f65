"""The DABA objective as a differentiable PyTorch function.

``objective(d, cams, lms, uv)`` sets the pixels and the iterate of the library context ``d``
and returns F(x) in pixel^2 (Eq. Fobj) as a 0-dim float64 tensor whose backward pass returns
dF/dcams (M x 9), dF/dlms (N x 3) and dF/duv (nnz x 2). Forward and gradient come from one
call of the library's adjoint kernels (``daba_objective_grad``); PyTorch only holds the
buffers. The observation list (which camera sees which landmark) is the one fixed by
``d.set_observations``.
"""
from __future__ import annotations

import torch


def _f64(x, name):
    if not isinstance(x, torch.Tensor) or x.dtype != torch.float64 or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    return x.detach().contiguous()


class DabaObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, cams, lms, uv, handle):
        cams_, lms_, uv_ = _f64(cams, "cams"), _f64(lms, "lms"), _f64(uv, "uv")
        stream = torch.cuda.current_stream().cuda_stream
        handle.set_state(cams_, lms_, stream=stream)
        handle.set_pixels(uv_, stream=stream)
        F = torch.zeros(1, dtype=torch.float64, device=cams.device)
        g_cams, g_lms, g_uv = torch.empty_like(cams_), torch.empty_like(lms_), torch.empty_like(uv_)
        handle.objective_grad(F, g_cams, g_lms, g_uv, stream=stream)
        ctx.save_for_backward(g_cams, g_lms, g_uv)
        return F[0]

    @staticmethod
    def backward(ctx, gF):
        g_cams, g_lms, g_uv = ctx.saved_tensors
        return gF * g_cams, gF * g_lms, gF * g_uv, None


def objective(handle, cams, lms, uv):
    """F(x) of the library context ``handle`` at (cams, lms, uv), differentiable in all three."""
    return DabaObjective.apply(cams, lms, uv, handle)
