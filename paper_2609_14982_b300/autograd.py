"""Slowness -> receiver traveltimes as a differentiable PyTorch function.

forward:  T_a = state solve (eik_forward) for every source, then receiver sampling P_a.
backward: the adjoint of the frozen tangent (Sec. 4.4, Eq. source-transpose, slowness
          model, D = 0): grad_s = sum_a C_a^T A_a^-T P_a^T grad_d_a, run by
          tangent_apply_T on the frozen state of the same slowness.
The frozen state S_a is kept from forward to backward when it fits the memory budget;
otherwise backward recomputes it (state solve and tangent_build again), source chunk
by source chunk.  The tangent is the derivative of the frozen transport, which the
paper discretizes separately from the nonlinear state (Sec. 3.2), so it agrees with
finite differences of forward only to discretization accuracy.
"""
from __future__ import annotations

import torch

from . import eik

BYTES_PER_SOURCE_NODE = 160    # structure + weights + workspaces of one (source, node), upper estimate


def tangent_bytes(S: int, N: int) -> int:
    return int(S) * int(N) * BYTES_PER_SOURCE_NODE


class StateCache:
    """The traveltimes of the last forward pass, so that the next state solve of the same
    sources starts from them (eik_forward_warm): in an inversion loop the state of outer
    iteration k+1 is solved from that of iteration k.  `cycles` records the sweep cycles
    each forward pass used."""

    def __init__(self):
        self.T = None
        self.key = None
        self.cycles = []


class SlownessToTraveltime(torch.autograd.Function):
    @staticmethod
    def forward(ctx, s, dgrid, src, rec, opts, budget_bytes, cache=None):
        src = [int(a) for a in src]
        key = (id(dgrid), tuple(src))
        if cache is not None and cache.T is not None and cache.key == key:
            T, cyc = eik.eik_forward(dgrid, s, src, opts, T_init=cache.T)
        else:
            T, cyc = eik.eik_forward(dgrid, s, src, opts)
        if cache is not None:
            cache.T, cache.key = T.detach().clone(), key
            cache.cycles.append(cyc)
        keep = tangent_bytes(len(src), dgrid.N) <= budget_bytes
        if keep:
            tan = eik.Tangent(dgrid, T, s, src, rec=rec, opts=opts)
            d = tan.sample(T)
            ctx.tan = tan
        else:
            chunk = max(1, budget_bytes // tangent_bytes(1, dgrid.N))
            outs = []
            for c0 in range(0, len(src), chunk):
                tan = eik.Tangent(dgrid, T[c0:c0 + chunk].contiguous(), s, src[c0:c0 + chunk], rec=rec, opts=opts)
                outs.append(tan.sample(T[c0:c0 + chunk].contiguous()))
                tan.free()
            d = torch.cat(outs)
            ctx.tan = None
            ctx.chunk = chunk
        ctx.dgrid, ctx.src, ctx.rec, ctx.opts = dgrid, src, rec, opts
        ctx.recomputed = not keep
        ctx.save_for_backward(s)
        return d

    @staticmethod
    def backward(ctx, grad_d):
        (s,) = ctx.saved_tensors
        y = grad_d.detach().to(torch.float64).contiguous().unsqueeze(-1)
        if ctx.tan is not None:
            g, _ = ctx.tan.apply_T(y, sum_sources=True)
            ctx.tan.free()
            ctx.tan = None
            return g[:, 0], None, None, None, None, None, None
        # recompute the frozen state chunk by chunk; each chunk's source sum is added to
        # the gradient by the library (tangent_apply_T with sum_sources = 2)
        total = torch.zeros((ctx.dgrid.N, 1), dtype=torch.float64, device=s.device)
        for c0 in range(0, len(ctx.src), ctx.chunk):
            part = ctx.src[c0:c0 + ctx.chunk]
            T, _ = eik.eik_forward(ctx.dgrid, s, part, ctx.opts)
            tan = eik.Tangent(ctx.dgrid, T, s, part, rec=ctx.rec, opts=ctx.opts)
            tan.apply_T(y[c0:c0 + ctx.chunk].contiguous(), sum_sources=True, g=total, accumulate=True)
            tan.free()
        return total[:, 0], None, None, None, None, None, None


def slowness_to_traveltime(s: torch.Tensor, dgrid, src, rec, opts=None, budget_bytes: int | None = None,
                           cache: StateCache | None = None):
    """Receiver traveltimes [S, n_rec] of slowness s [N] (FP64, on the device).
    budget_bytes bounds the memory kept for backward (default: half the free memory);
    with a StateCache the state solve starts from the previous call's traveltimes."""
    if budget_bytes is None:
        free, _ = torch.cuda.mem_get_info()
        budget_bytes = free // 2
    return SlownessToTraveltime.apply(s, dgrid, src, rec, opts or eik.default_opts(), int(budget_bytes), cache)
