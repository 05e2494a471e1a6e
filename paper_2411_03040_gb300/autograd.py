"""torch.autograd.Function around mgt_image and its hand-written adjoint.

    I = ImageFunction.apply(log_T, log_n_spec, vel, model, direction, npx, npy,
                            nfreq, fmin, fmax)

log_T [N], log_n_spec [N] and vel [N][3] are float64 CUDA tensors; the
result is the f32 image [nfreq][npy][npx].  The forward pass writes the fields
into the model (mgt_set_point_fields, populations kept as fractions of
n_spec) and calls mgt_image; the backward pass calls mgt_image_adjoint.  The
exponentials of the log fields are argument preparation; the image and its
gradient are computed by the CUDA library.
"""
from __future__ import annotations

import torch

from . import mgt


class ImageFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_T, log_n, vel, model, direction, npx, npy, nfreq, fmin, fmax):
        stream = torch.cuda.current_stream()
        T = torch.exp(log_T.detach()).contiguous()
        n = torch.exp(log_n.detach()).contiguous()
        v = vel.detach().contiguous()
        mgt.mgt_set_point_fields(model, T, n, v, stream=stream)
        out = torch.empty((nfreq, npy, npx), dtype=torch.float32, device=log_T.device)
        mgt.mgt_image(model, direction, npx, npy, nfreq, fmin, fmax, out=out, stream=stream)
        ctx.args = (model, direction, npx, npy, nfreq, fmin, fmax)
        ctx.N = log_T.shape[0]
        return out

    @staticmethod
    def backward(ctx, grad_out):
        model, direction, npx, npy, nfreq, fmin, fmax = ctx.args
        dev = grad_out.device
        g = grad_out.contiguous().to(torch.float32)
        gT = torch.empty(ctx.N, dtype=torch.float64, device=dev)
        gn = torch.empty(ctx.N, dtype=torch.float64, device=dev)
        gv = torch.empty((ctx.N, 3), dtype=torch.float64, device=dev)
        mgt.mgt_image_adjoint(model, direction, npx, npy, nfreq, fmin, fmax, g, gT, gn, gv,
                              stream=torch.cuda.current_stream())
        return gT, gn, gv, None, None, None, None, None, None, None
