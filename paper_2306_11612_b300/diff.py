"""Differentiable dynamic volume lines: gradients for automatic TF tuning.

``AlphaMeans.apply(dvl, ctrl, **params)`` maps alpha control points
``ctrl`` (M, K) -- a CUDA tensor in [0, 1] -- to the per-pixel mean alpha
(M, W) of a DVL update; its backward pass returns dL/dctrl through the
library's adjoint kernel, with the cell-to-pixel assignment and the cells'
TF entries held fixed at the forward pass (they are piecewise constant in
the control points).  Only marshalling happens here: the tables, the update,
the means and the adjoint all run in the library's CUDA kernels.
"""
from __future__ import annotations

import torch


class AlphaMeans(torch.autograd.Function):
    @staticmethod
    def forward(ctx, dvl, ctrl, n_entries=256, P=1.0, min_importance=0.025, width=1024, min_imp_mode=0,
                vmax_mode=0, width_mode=0):
        if not ctrl.is_cuda:
            raise ValueError("ctrl must be a CUDA tensor")
        ctrl = ctrl.detach().float().contiguous()
        cur, lib_stream = torch.cuda.current_stream(), dvl.torch_stream()
        lib_stream.wait_stream(cur)                   # ctrl is read on the library's stream
        out = torch.empty((dvl.M, width), dtype=torch.float32, device=ctrl.device)
        dvl.set_tf_ctrl(ctrl, n_entries)
        dvl.update(P=P, min_importance=min_importance, width=width, min_imp_mode=min_imp_mode,
                   vmax_mode=vmax_mode, width_mode=width_mode, want_alpha=1)
        dvl.read_alpha_means(out)                     # device copy, ordered on the library's stream
        cur.wait_stream(lib_stream)                   # later uses (and frees) of ctrl / out follow it
        ctx.dvl = dvl
        ctx.K = ctrl.shape[1]
        return out

    @staticmethod
    def backward(ctx, grad_out):
        g = grad_out.detach().float().contiguous()
        cur, lib_stream = torch.cuda.current_stream(), ctx.dvl.torch_stream()
        lib_stream.wait_stream(cur)
        grad = torch.empty((ctx.dvl.M, ctx.K), dtype=torch.float32, device=g.device)
        ctx.dvl.backward(g, grad)                     # device in and out: asynchronous
        cur.wait_stream(lib_stream)
        return (None, grad) + (None,) * 7


def alpha_means(dvl, ctrl, **params):
    """Per-pixel mean alpha (M, W) as a differentiable function of ctrl (M, K)."""
    return AlphaMeans.apply(dvl, ctrl, params.get("n_entries", 256), params.get("P", 1.0),
                            params.get("min_importance", 0.025), params.get("width", 1024),
                            params.get("min_imp_mode", 0), params.get("vmax_mode", 0),
                            params.get("width_mode", 0))
