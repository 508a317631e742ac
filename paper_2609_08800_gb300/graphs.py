"""CUDA graphs per horizon chunk.

A chunk -- `steps` forward steps recording the tape, optionally followed by the
`steps` adjoint steps back through it -- is captured once into a CUDA graph over
static device buffers and then replayed: one graph launch replaces 2 x steps kernel
launches and their host round trips (what matters for small batches and the serving
loop).  Inputs are copied into the static buffers before a replay; outputs are read
from them after.
"""
from __future__ import annotations

import torch


class ChunkGraph:
    def __init__(self, ctx, steps, h, with_adjoint=True, stream=None):
        if ctx.tape_slots < steps:
            raise ValueError("the context needs one tape slot per step of the chunk")
        self.ctx, self.steps, self.h, self.with_adjoint = ctx, steps, h, with_adjoint
        dev, dt, ns, W = "cuda", ctx.dtype, ctx.n_state, ctx.ld
        self.s0 = torch.zeros(ns, W, dtype=dt, device=dev)
        self.controls = torch.zeros(steps, max(ctx.n_servo, 1), W, dtype=dt, device=dev)
        self.gT = torch.zeros(ns, W, dtype=dt, device=dev)
        self.states = torch.zeros(steps + 1, ns, W, dtype=dt, device=dev)
        self.grads = torch.zeros(steps + 1, ns, W, dtype=dt, device=dev)
        self.dcontrols = torch.zeros(steps, max(ctx.n_servo, 1), W, dtype=dt, device=dev)
        self.status = torch.zeros(steps, W, dtype=torch.int32, device=dev)
        self.iters = torch.zeros(steps, W, dtype=torch.int32, device=dev)
        self.graph = torch.cuda.CUDAGraph()
        side = stream or torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self._body()                     # warm-up: kernel attributes, lazy loading
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        with torch.cuda.graph(self.graph):
            self._body()

    def _body(self):
        ctx = self.ctx
        self.states[0].copy_(self.s0)
        for t in range(self.steps):
            ctx.ostrich_step(self.states[t], self.controls[t], self.h, self.states[t + 1], None, None,
                             self.status[t], self.iters[t], tape_slot=t)
        if self.with_adjoint:
            self.grads[self.steps].copy_(self.gT)
            for t in reversed(range(self.steps)):
                ctx.ostrich_adjoint(t, self.grads[t + 1], self.h, self.grads[t], self.dcontrols[t])

    def replay(self, s0=None, controls=None, gT=None):
        if s0 is not None:
            self.s0.copy_(s0)
        if controls is not None:
            self.controls[:, :controls.shape[1]].copy_(controls)
        if gT is not None:
            self.gT.copy_(gT)
        self.graph.replay()
        return self.states, self.grads, self.dcontrols
