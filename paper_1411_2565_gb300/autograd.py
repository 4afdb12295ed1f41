"""torch.autograd.Function over the LLG time stepper.

``llg(m0, hext, ms, g, n, dt)`` returns m after ``n`` Euler steps of film ``g``
(a ``Grace``) from ``m0`` with a per-cell applied field ``hext`` (3N, A/m) and a per-cell
saturation magnetisation ``ms`` (N, A/m).  The forward pass keeps every
``ckpt_every``-th state (grace_step_checkpointed); the backward pass calls the
hand-written discrete adjoint from those checkpoints (grace_backward_checkpointed):
states are re-computed between checkpoints, and the gradients with respect to m0, hext
and ms come back from the CUDA kernels.  All tensors are flat FP32 on the film's device.
"""
from __future__ import annotations

import torch


class LLGFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m0, hext, ms, g, n, dt, ckpt_every):
        m0, hext, ms = m0.detach().contiguous(), hext.detach().contiguous(), ms.detach().contiguous()
        g.set_ms_field(ms)
        g.set_hext_field(hext)
        g.set_m(m0)
        tape = g.step_checkpointed(n, dt, ckpt_every)
        mT = g.get_m()
        ctx.save_for_backward(m0, hext, ms)
        ctx.g, ctx.n, ctx.dt, ctx.ckpt, ctx.tape = g, n, dt, ckpt_every, tape
        return mT

    @staticmethod
    def backward(ctx, grad_mT):
        m0, hext, ms = ctx.saved_tensors
        g = ctx.g
        g.set_ms_field(ms)
        g.set_hext_field(hext)
        g_h = torch.zeros_like(hext)
        g_ms = torch.zeros_like(ms)
        g_m0 = g.backward(grad_mT.contiguous().float(), ctx.n, ctx.dt, ctx.ckpt, g_h, g_ms, True, tape=ctx.tape)
        ctx.tape = None
        return g_m0, g_h, g_ms, None, None, None, None


def llg(m0, hext, ms, g, n: int, dt: float, ckpt_every: int = 64):
    return LLGFunction.apply(m0, hext, ms, g, n, dt, ckpt_every)
