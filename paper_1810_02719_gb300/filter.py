"""Differentiable block low-pass filter X -> U U^T X as a torch.autograd.Function.

Forward and backward both run in the library's CUDA kernels (bsp_filter_forward
and bsp_filter_backward); torch provides the device buffers and the stream.
The mesh must be created with weight_mode = BSP_W_EDGE; the weights passed to
``apply`` are installed with bsp_set_edge_weights before the forward pass.  A
backward pass uses the checkpoints of the mesh's most recent forward pass.
"""
from __future__ import annotations

import torch

from . import bsp


class BlockLowPass(torch.autograd.Function):
    """y = U U^T x per block, U from t_max unrolled OI steps on L(w) (starts detached)."""

    @staticmethod
    def forward(ctx, x, w, mesh, c, t_max, V0_roots):
        if not (x.is_cuda and w.is_cuda):
            raise ValueError("BlockLowPass runs on CUDA tensors only")
        x = x.detach().contiguous()
        bsp.bsp_set_edge_weights(mesh, w.detach().contiguous())
        out = torch.empty_like(x)
        stream = torch.cuda.current_stream(x.device)
        bsp.bsp_filter_forward(mesh, c, t_max, V0_roots, x, out, stream)
        ctx.mesh = mesh
        ctx.n_edges = w.shape[0]
        ctx.save_for_backward(x)
        return out

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        g = g.contiguous()
        dx = torch.empty_like(x)
        dw = torch.empty(ctx.n_edges, dtype=x.dtype, device=x.device)
        stream = torch.cuda.current_stream(x.device)
        bsp.bsp_filter_backward(ctx.mesh, g, x, dx, dw, stream)
        return dx, dw, None, None, None, None


def block_low_pass(x, w, mesh, c, t_max, V0_roots):
    return BlockLowPass.apply(x, w, mesh, c, t_max, V0_roots)
