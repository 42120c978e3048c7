"""torch.autograd wrapper of the continuous peak and its adjoint (ccst_peak_continuous /
ccst_backward). Argument marshalling only: the forward and backward passes run in the
library's kernels."""
from __future__ import annotations

import torch

from . import ccst as C


class ContinuousPeak(torch.autograd.Function):
    """(dx, dy) of the continuous peak of every frame against the tracker's reference.

    Inputs: frames (n, H, W) float32 CUDA tensor, ref (H, W) float32 CUDA tensor holding the
    tracker's reference (the leaf that receives dL/dE; its values are not read).
    Output: (n, 2) float64 (dx, dy). The grid peak that starts Newton's method comes from a
    ccst_track of the same frames."""

    @staticmethod
    def forward(ctx, frames, ref, tracker):
        n = frames.shape[0]
        frames = frames.contiguous()
        rec = tracker.empty_results(n)
        for s in range(0, n, tracker.max_batch):
            e = min(n, s + tracker.max_batch)
            C.ccst_track(tracker.ctx, frames[s:e], e - s, 0, rec[s:e])
        peak = torch.empty((n, 2), dtype=torch.float64, device=frames.device)
        status = torch.empty((n,), dtype=torch.int32, device=frames.device)
        C.ccst_peak_continuous(tracker.ctx, frames, n, 0, rec, peak, status)
        ctx.save_for_backward(frames, rec)
        ctx.tracker = tracker
        ctx.mark_non_differentiable(status)
        return peak, status

    @staticmethod
    def backward(ctx, g_peak, g_status):
        frames, rec = ctx.saved_tensors
        t = ctx.tracker
        n, H, W = frames.shape
        g = g_peak.to(torch.float32).contiguous()
        g_frames = torch.empty((n, H, W), dtype=torch.float32, device=frames.device) \
            if ctx.needs_input_grad[0] else None
        g_ref = torch.empty((H, W), dtype=torch.float32, device=frames.device) if ctx.needs_input_grad[1] else None
        C.ccst_backward(t.ctx, frames, n, 0, rec, g, g_frames, g_ref)
        return g_frames, g_ref, None


def continuous_peak(tracker, frames, ref):
    """Differentiable (dx, dy) and status (0 = a proper extremum found) of every frame."""
    return ContinuousPeak.apply(frames, ref, tracker)
