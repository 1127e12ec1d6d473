"""Differentiable LP layer: K unrolled iterations of restarted reflected-Halpern PDHG over a batch
of LPs, with the restart schedule and the primal weight frozen from a forward solve, as a
torch.autograd.Function.  Forward and backward run in the library's kernels
(include/lp_diff.h); this module only marshals tensors.

The gradient is the exact derivative of the unrolled K-step map (piecewise affine between
restarts), not the derivative of the LP solution.  At a nondegenerate vertex the LP solution is
locally constant in c, so its derivative in c is 0; the unrolled map's derivative tends to it as
the iterates settle, and it is informative for the bounds (b) where the solution moves.
"""
from __future__ import annotations

import numpy as np
import torch

from . import BatchSolver


class UnrolledLPBatch:
    """Holds the batch (its matrices are fixed) and applies the differentiable map to new
    objectives and bounds: ``x, y = layer(c, l_c, u_c, l_v, u_v)`` with CUDA float64 tensors
    concatenated over the instances in their original order.  ``params`` go to the batch
    (lp_params fields).  Defaults for the layer: instances with at most 65536 nonzeros count as
    small and run their unrolled iterations (and the traced solve) on clusters of CTAs with
    cluster barriers, the others on the grid kernels; the tile schedule is lane_target 16,
    tile_rows 8, the fastest measured for the unrolled kernels."""

    def __init__(self, lps, K: int = 2000, checkpoint_every: int = 100, **params):
        params.setdefault("precision", 0)
        params.setdefault("lane_target", 16)
        params.setdefault("tile_rows", 8)
        params.setdefault("batch_local_nnz", 1 << 16)
        self.batch = BatchSolver(lps, **params)
        self.K, self.C = int(K), int(checkpoint_every)
        self.sum_n = int(sum(lp.n for lp in lps))
        self.sum_m = int(sum(lp.m for lp in lps))

    def __call__(self, c, l_c, u_c, l_v, u_v):
        return _Unrolled.apply(self, c, l_c, u_c, l_v, u_v)

    def close(self):
        self.batch.close()


class _Unrolled(torch.autograd.Function):
    @staticmethod
    def forward(ctx, layer, c, l_c, u_c, l_v, u_v):
        ts = [t.detach().to(torch.float64).contiguous() for t in (c, l_c, u_c, l_v, u_v)]
        for t in ts:
            if not t.is_cuda:
                raise ValueError("UnrolledLPBatch needs CUDA float64 tensors")
        stream = torch.cuda.current_stream().cuda_stream
        torch.cuda.current_stream().synchronize()
        layer.batch.set_data(*ts)
        x = torch.empty(layer.sum_n, dtype=torch.float64, device=ts[0].device)
        y = torch.empty(layer.sum_m, dtype=torch.float64, device=ts[0].device)
        layer.batch.unroll(layer.K, layer.C, x, y, stream)
        ctx.layer = layer
        ctx.dev = ts[0].device
        return x, y

    @staticmethod
    def backward(ctx, gx, gy):
        layer = ctx.layer
        need = ctx.needs_input_grad[1:]
        shapes = (layer.sum_n, layer.sum_m, layer.sum_m, layer.sum_n, layer.sum_n)
        grads = [torch.zeros(n, dtype=torch.float64, device=ctx.dev) if w else None for n, w in zip(shapes, need)]
        gx = None if gx is None else gx.to(torch.float64).contiguous()
        gy = None if gy is None else gy.to(torch.float64).contiguous()
        layer.batch.unroll_vjp(gx, gy, *grads, stream=torch.cuda.current_stream().cuda_stream)
        return (None, *grads)
