"""The DABA objective as a differentiable PyTorch function.

``objective(d, cams, lms, uv)`` sets the pixels and the iterate of the library context ``d``
and returns F(x) in pixel^2 (Eq. Fobj) as a 0-dim float64 tensor whose backward pass returns
dF/dcams (M x 9), dF/dlms (N x 3) and dF/duv (nnz x 2). Forward and gradient come from one
call of the library's adjoint kernels (``daba_objective_grad``); PyTorch only holds the
buffers. The observation list (which camera sees which landmark) is the one fixed by
``d.set_observations``.

``unrolled(d, cams, lms, uv, K)`` runs K iterations of Algorithm 1 from (cams, lms) with the
pixels uv and returns the boundary state (cams_K, lms_K); its backward pass is the
vector-Jacobian product of the K iterations (``daba_unrolled_grad``: adjoint kernels, states
kept every 10 iterations, restart decisions held at those of the run). FP64 contexts only.
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


class DabaUnrolled(torch.autograd.Function):
    @staticmethod
    def forward(ctx, cams, lms, uv, handle, K):
        cams_, lms_, uv_ = _f64(cams, "cams"), _f64(lms, "lms"), _f64(uv, "uv")
        stream = torch.cuda.current_stream().cuda_stream
        handle.set_state(cams_, lms_, stream=stream)
        handle.set_pixels(uv_, stream=stream)
        handle.run(K, stream=stream)
        out_c, out_l = torch.empty_like(cams_), torch.empty_like(lms_)
        handle.get_state(out_c, out_l, stream=stream)
        ctx.save_for_backward(cams_, lms_, uv_)
        ctx.handle, ctx.K = handle, K
        return out_c, out_l

    @staticmethod
    def backward(ctx, g_out_c, g_out_l):
        cams_, lms_, uv_ = ctx.saved_tensors
        handle = ctx.handle
        stream = torch.cuda.current_stream().cuda_stream
        seed_c = torch.zeros_like(cams_) if g_out_c is None else g_out_c.to(torch.float64).contiguous()
        seed_l = torch.zeros_like(lms_) if g_out_l is None else g_out_l.to(torch.float64).contiguous()
        # the product is taken from the input state, which the context no longer holds
        handle.set_state(cams_, lms_, stream=stream)
        handle.set_pixels(uv_, stream=stream)
        g_c, g_l, g_u = torch.empty_like(cams_), torch.empty_like(lms_), torch.empty_like(uv_)
        handle.unrolled_grad(ctx.K, seed_c, seed_l, g_c, g_l, g_u, stream=stream)
        return g_c, g_l, g_u, None, None


def unrolled(handle, cams, lms, uv, K):
    """State (cams_K, lms_K) after K iterations of the library context ``handle`` from
    (cams, lms) with pixels uv, differentiable in all three inputs."""
    return DabaUnrolled.apply(cams, lms, uv, handle, int(K))
