"""torch.autograd.Function over gbt_sum / gbt_sum_backward.

    p = gbs_field(trace, recv, freqs, beam_b, gamma, ray_weight, ...)   # complex64 [F, Nr]
    loss = (p - target).abs().pow(2).sum(); loss.backward()

Differentiable inputs: ``gamma`` (per-material reflection coefficients,
float32), ``ray_weight`` (per-ray source weights, float32, optional) and
``beam_b`` (per-frequency beam parameter, float64 tensor on the device).  The
cull mask and window are held fixed: the summand is differentiated where it is
kept.  The backward pass recomputes every kept contribution in the library's
kernel (nothing is stored per receiver and segment).  For a real loss torch
hands the backward ``g = dL/dRe p + i dL/dIm p``, which is the convention of
gbt_sum_backward, so the gradients are ``sum Re(conj(g) dp/dtheta)``.  Optional
propagation losses (``absorption`` per frequency in Np/m, ``flow_resistivity`` per
material) enter the field and its gradients but are not differentiated.  The backward
pass ends by reading the library's device status word (gbt_sync on the current
stream), so a kernel that flagged a problem (a bounded wait that ran out) raises
instead of leaving a partial gradient.
"""
from __future__ import annotations

import torch

from . import gbt as G


class GBTSum(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gamma, ray_weight, beam_b, trace, recv, freqs, order, window, cutoff,
                tile_cull=False, absorption=None, flow_resistivity=None):
        b = [float(v) for v in beam_b.detach().cpu().tolist()]
        p = G.gbs_sum(trace, recv, list(freqs), b, gamma.detach().contiguous(),
                      ray_weight=None if ray_weight is None else ray_weight.detach().contiguous(),
                      order=order, window=window, cutoff=cutoff, tile_cull=tile_cull,
                      absorption=absorption, flow_resistivity=flow_resistivity)
        ctx.absorption, ctx.flow_resistivity = absorption, flow_resistivity
        ctx.save_for_backward(gamma, ray_weight if ray_weight is not None else torch.empty(0))
        ctx.has_w = ray_weight is not None
        ctx.trace, ctx.recv, ctx.freqs, ctx.b, ctx.order = trace, recv, list(freqs), b, order
        ctx.window, ctx.cutoff, ctx.tile_cull = window, cutoff, tile_cull
        ctx.b_dtype, ctx.b_device = beam_b.dtype, beam_b.device
        return p

    @staticmethod
    def backward(ctx, grad_p):
        gamma, w = ctx.saved_tensors
        w = w if ctx.has_w else None
        need_w = ctx.needs_input_grad[1]
        need_b = ctx.needs_input_grad[2]
        dg, dw, db = G.gbs_sum_backward(ctx.trace, ctx.recv, ctx.freqs, ctx.b,
                                        gamma.detach().contiguous(),
                                        grad_p.to(torch.complex64).contiguous(),
                                        ray_weight=None if w is None else w.detach().contiguous(),
                                        order=ctx.order, window=ctx.window, cutoff=ctx.cutoff,
                                        need_weight=need_w, need_b=need_b,
                                        tile_cull=ctx.tile_cull, absorption=ctx.absorption,
                                        flow_resistivity=ctx.flow_resistivity)
        G.gbt_sync(G._stream_ptr())    # raises if a kernel of this step flagged a problem
        gw = dw if (need_w and w is not None) else None
        gb = db.to(device=ctx.b_device, dtype=ctx.b_dtype) if need_b else None
        return (dg if ctx.needs_input_grad[0] else None, gw, gb,
                None, None, None, None, None, None, None, None, None)


def gbs_field(trace, recv, freqs, beam_b, gamma, ray_weight=None, order=None,
              window: int = G.WINDOW_LINE, cutoff: float = 16.0, tile_cull: bool = False,
              absorption=None, flow_resistivity=None):
    """Differentiable complex pressure p[f, r] (complex64); ``tile_cull`` runs forward and
    backward with the exact tile pre-cull."""
    if not torch.is_tensor(beam_b):
        beam_b = torch.tensor(list(beam_b), dtype=torch.float64, device=recv.device)
    ab = None if absorption is None else tuple(float(v) for v in absorption)
    return GBTSum.apply(gamma, ray_weight, beam_b, trace, recv, tuple(freqs), order, window,
                        float(cutoff), bool(tile_cull), ab, flow_resistivity)
