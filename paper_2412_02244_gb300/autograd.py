"""torch.autograd.Function wrappers of the differentiable k-means losses.

Both run entirely in libdkm's kernels (dkm_soft_forward / dkm_soft_backward
/ dkm_hard_sse / dkm_hard_sse_backward / dkm_soft_temperature); this module
only allocates the output tensors and routes the upstream gradient.

  SoftKMeansLoss.apply(points, init, offsets, tau, T) -> loss (B,) float64
      points  (n_total, d) float32 CUDA, clouds concatenated
      init    (B, k, d)    float32 CUDA, initial centroids
      offsets (B + 1,)     int64 (CPU), cloud b = points[offsets[b]:offsets[b+1]]
      tau     (B,)         float32 (CPU), temperature per cloud (a constant);
                           None = temperature(points, offsets)
      T       int          unrolled soft k-means steps
    Gradients flow to points and init.

  HardSSELoss.apply(points, centroids, offsets) -> loss (B,) float64
    Gradients flow to points and centroids.
"""
from __future__ import annotations

import torch

from . import dkm


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def temperature(points: torch.Tensor, offsets: torch.Tensor, frac: float = 0.01) -> torch.Tensor:
    """tau_b = frac x squared bounding-box diagonal of cloud b (CPU float32),
    computed on the GPU by dkm_soft_temperature."""
    offsets = offsets.to(torch.int64).cpu().contiguous()
    B = offsets.numel() - 1
    tau = torch.empty(B, dtype=torch.float32)
    dkm.dkm_soft_temperature(points.contiguous(), offsets, B, points.shape[1], tau, frac,
                             _stream())
    return tau


class SoftKMeansLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, points, init, offsets, tau, T: int):
        B, k, d = init.shape
        points = points.contiguous()
        init = init.contiguous()
        offsets = offsets.to(torch.int64).cpu().contiguous()
        if tau is None:
            tau = temperature(points, offsets)
        tau = tau.to(torch.float32).cpu().contiguous()
        ckpt = torch.empty((T + 1, B, k, d), dtype=torch.float32, device=points.device)
        loss = torch.empty(B, dtype=torch.float64, device=points.device)
        # per-step softmax statistics (O(n) per step) so the backward need not
        # recompute them; the n x k weights are never stored
        n_total = points.shape[0]
        stats = torch.empty((T, 2, n_total), dtype=torch.float32, device=points.device)
        norms = torch.empty((T, B, k), dtype=torch.float32, device=points.device)
        dkm.dkm_soft_forward(points, offsets, B, d, k, init, T, tau, ckpt, loss, _stream(),
                             stats=stats, norms=norms)
        ctx.save_for_backward(points, ckpt, stats, norms)
        ctx.meta = (offsets, tau, int(T), B, k, d)
        return loss

    @staticmethod
    def backward(ctx, gloss):
        points, ckpt, stats, norms = ctx.saved_tensors
        offsets, tau, T, B, k, d = ctx.meta
        gp = torch.empty_like(points)
        gi = torch.empty((B, k, d), dtype=torch.float32, device=points.device)
        dl = gloss.detach().to(torch.float64).contiguous()
        dkm.dkm_soft_backward(points, offsets, B, d, k, ckpt, T, tau, dl, gp, gi, _stream(),
                              stats=stats, norms=norms)
        return gp, gi, None, None, None


class HardSSELoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, points, centroids, offsets):
        B, k, d = centroids.shape
        points = points.contiguous()
        centroids = centroids.contiguous()
        offsets = offsets.to(torch.int64).cpu().contiguous()
        loss = torch.empty(B, dtype=torch.float64, device=points.device)
        labels = torch.empty(points.shape[0], dtype=torch.int32, device=points.device)
        dkm.dkm_hard_sse(points, offsets, B, d, k, centroids, labels, loss, None, None, _stream())
        ctx.save_for_backward(points, centroids, labels)
        ctx.offsets = offsets
        return loss

    @staticmethod
    def backward(ctx, gloss):
        points, centroids, labels = ctx.saved_tensors
        B, k, d = centroids.shape
        gp = torch.empty_like(points) if ctx.needs_input_grad[0] else None
        gc = torch.empty_like(centroids) if ctx.needs_input_grad[1] else None
        dl = gloss.detach().to(torch.float64).contiguous()
        dkm.dkm_hard_sse_backward(points, ctx.offsets, B, d, k, centroids, labels, dl, gp, gc,
                                  _stream())
        return gp, gc, None
