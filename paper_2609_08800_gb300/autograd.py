"""Differentiable rollouts: a torch.autograd.Function over a horizon of steps.

Forward runs T steps s_{t+1} = step(s_t, a_t); backward sweeps the IFT adjoint of
each step in reverse (Sec. III-D), adding the loss's direct gradient of every state on
the way.  With checkpointing the forward records nothing but the states; the backward
recomputes each segment's steps into a tape of `segment` slots just before sweeping
it, so device memory for the factors is O(segment) instead of O(T).  The kernels are
deterministic, so the checkpointed gradient is bit-identical to the plain one.

The stepping engine is a small object with `step(s_in, a, slot) -> s_out` and
`adjoint(slot, g) -> (dL/ds_in, dL/da)`; the product engine is `CudaEngine` (libostrich).
"""
from __future__ import annotations

import math

import torch

from .ostrich import Context


class CudaEngine:
    """libostrich context over W worlds with `slots` tape slots."""

    def __init__(self, scene, cfg, n_worlds, h, slots, dtype="f32", threads=None):
        self.ctx = Context(scene, cfg, n_worlds, dtype=dtype, tape_slots=slots, threads=threads)
        self.h = h
        self.dtype = self.ctx.dtype
        self.slots = slots
        self.n_state, self.n_servo, self.ld = self.ctx.n_state, self.ctx.n_servo, self.ctx.ld

    def step(self, s_in, a, slot):
        out = torch.empty_like(s_in)
        self.ctx.ostrich_step(s_in, a, self.h, out, tape_slot=slot)
        return out

    def adjoint(self, slot, g):
        ds = torch.empty_like(g)
        du = torch.empty(max(self.n_servo, 1), self.ld, dtype=g.dtype, device=g.device)
        self.ctx.ostrich_adjoint(slot, g, self.h, ds, du)
        return ds, du[:self.n_servo]

    def clear(self):
        self.ctx.ostrich_tape_clear()

    def close(self):
        self.ctx.close()


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(fctx, s0, controls, engine, segment):
        T = controls.shape[0]
        ckpt = segment is not None and segment < T
        states = [s0]
        with torch.no_grad():
            for t in range(T):
                slot = -1 if ckpt else t
                states.append(engine.step(states[t], controls[t], slot))
        traj = torch.stack(states)
        fctx.engine, fctx.segment, fctx.ckpt = engine, segment, ckpt
        fctx.save_for_backward(traj, controls)
        return traj

    @staticmethod
    def backward(fctx, gtraj):
        traj, controls = fctx.saved_tensors
        engine, ckpt = fctx.engine, fctx.ckpt
        T = controls.shape[0]
        seg = fctx.segment if ckpt else T
        g = gtraj[T].contiguous()
        gctl = torch.zeros_like(controls)
        n_seg = math.ceil(T / seg)
        for k in reversed(range(n_seg)):
            t0, t1 = k * seg, min(T, (k + 1) * seg)
            if ckpt:
                # recompute the segment into slots 0..t1-t0-1 (deterministic: same factors)
                with torch.no_grad():
                    s = traj[t0]
                    for t in range(t0, t1):
                        s = engine.step(s, controls[t], t - t0)
            for t in reversed(range(t0, t1)):
                slot = t - t0 if ckpt else t
                ds, du = engine.adjoint(slot, g)
                gctl[t] = du
                g = ds + gtraj[t]
        return g, gctl, None, None


def rollout(s0, controls, engine, segment=None):
    """States [T + 1, n_state, ld] of a T-step rollout, differentiable in s0 and controls
    [T, n_servo, ld].  segment: checkpoint every `segment` steps (None: keep every
    step's factor on the tape; the engine then needs T slots)."""
    return _Rollout.apply(s0, controls, engine, segment)
