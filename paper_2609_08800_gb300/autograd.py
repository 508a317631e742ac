"""Differentiable rollouts: a torch.autograd.Function over a horizon of steps.

Forward runs T steps s_{t+1} = step(s_t, a_t); backward sweeps the IFT adjoint of
each step in reverse (Sec. III-D), adding the loss's direct gradient of every state on
the way.  With checkpointing the forward keeps the states and records only the last
segment's steps into the tape of `segment` slots; the backward sweeps that segment
straight from the tape (when nothing has recorded into the engine's tape since) and
recomputes each earlier segment's steps into the same slots just before sweeping it,
so device memory for the factors is O(segment) instead of O(T).  The kernels are
deterministic, so the checkpointed gradient is bit-identical to the plain one.

The stepping engine is a small object with `step(s_in, a, slot) -> s_out` and
`adjoint(slot, g) -> (dL/ds_in, dL/da)`; the product engine is `CudaEngine` (libostrich).

Physical parameters (Eq. (17) with xi = theta): pass `theta`, the scene's parameter
vector from `engine.theta()` -- servo gains k_p (servo order), body masses, body-frame
principal moments (body-major) -- and the backward also returns dL/dtheta, summed over
the steps of the horizon and over the worlds (the parameters are shared).  The engine
then needs `adjoint_params(slot, g) -> (dL/ds_in, dL/da, dL/dtheta per world [P, W])`.
The values of `theta` are the scene's own: the rollout checks them and does not
re-parameterise the scene.
"""
from __future__ import annotations

import math

import torch

from .ostrich import Context


class CudaEngine:
    """libostrich context over W worlds with `slots` tape slots."""

    def __init__(self, scene, cfg, n_worlds, h, slots, dtype="f32", threads=None):
        self.scene = scene
        self.ctx = Context(scene, cfg, n_worlds, dtype=dtype, tape_slots=slots, threads=threads)
        self.h = h
        self.dtype = self.ctx.dtype
        self.slots = slots
        self.n_state, self.n_servo, self.ld = self.ctx.n_state, self.ctx.n_servo, self.ctx.ld
        # counts the recordings into the tape (steps with a slot, clears): a rollout's
        # backward reuses the slots its forward recorded only while the count is unchanged
        self.tape_epoch = 0

    def step(self, s_in, a, slot):
        out = torch.empty_like(s_in)
        self.ctx.ostrich_step(s_in, a, self.h, out, tape_slot=slot)
        if slot >= 0:
            self.tape_epoch += 1
        return out

    def adjoint(self, slot, g):
        ds = torch.empty_like(g)
        du = torch.empty(max(self.n_servo, 1), self.ld, dtype=g.dtype, device=g.device)
        self.ctx.ostrich_adjoint(slot, g, self.h, ds, du)
        return ds, du[:self.n_servo]

    def adjoint_params(self, slot, g):
        ds, du, dkp, dm, di = self.ctx.adjoint_params(slot, g, self.h)
        return ds, du, torch.cat([dkp, dm, di.reshape(-1, di.shape[-1])], 0)

    def theta(self):
        return scene_theta(self.scene, dtype=self.dtype)

    def clear(self):
        self.ctx.ostrich_tape_clear()
        self.tape_epoch += 1

    def close(self):
        self.ctx.close()


def scene_theta(scene, dtype=torch.float64):
    """The scene's physical parameters in the order of the parameter gradients: servo
    gains k_p (joints with a servo, in joint order), body masses, body-frame principal
    moments (body-major, 3 per body)."""
    vals = [j.kp for j in scene.joints if j.kp > 0]
    vals += [b.mass for b in scene.bodies]
    for b in scene.bodies:
        vals += list(b.inertia)
    return torch.tensor(vals, dtype=dtype)


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(fctx, s0, controls, theta, engine, segment):
        T = controls.shape[0]
        ckpt = segment is not None and segment < T
        # with checkpointing, the last segment's steps are recorded now (slots 0, 1, ...),
        # so that the backward need not recompute them
        t_last = ((T - 1) // segment) * segment if ckpt else 0
        states = [s0]
        with torch.no_grad():
            for t in range(T):
                slot = (t - t_last if t >= t_last else -1) if ckpt else t
                states.append(engine.step(states[t], controls[t], slot))
        traj = torch.stack(states)
        fctx.engine, fctx.segment, fctx.ckpt = engine, segment, ckpt
        fctx.tape_epoch = getattr(engine, "tape_epoch", None)
        fctx.with_theta = theta is not None
        fctx.theta_shape = None if theta is None else theta.shape
        fctx.theta_dtype = None if theta is None else theta.dtype
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
        gth = None
        n_seg = math.ceil(T / seg)
        for k in reversed(range(n_seg)):
            t0, t1 = k * seg, min(T, (k + 1) * seg)
            # the last segment is still on the tape if nothing recorded into it since the
            # forward (an engine without a recording count always recomputes)
            taped = k == n_seg - 1 and fctx.tape_epoch is not None \
                and getattr(engine, "tape_epoch", None) == fctx.tape_epoch
            if ckpt and not taped:
                # recompute the segment into slots 0..t1-t0-1 (deterministic: same factors)
                with torch.no_grad():
                    s = traj[t0]
                    for t in range(t0, t1):
                        s = engine.step(s, controls[t], t - t0)
            for t in reversed(range(t0, t1)):
                slot = t - t0 if ckpt else t
                if fctx.with_theta:
                    ds, du, dth = engine.adjoint_params(slot, g)
                    step_th = dth.sum(1)
                    gth = step_th if gth is None else gth + step_th
                else:
                    ds, du = engine.adjoint(slot, g)
                gctl[t] = du
                g = ds + gtraj[t]
        if gth is not None:
            gth = gth.to(device="cpu", dtype=fctx.theta_dtype).reshape(fctx.theta_shape)
        return g, gctl, gth, None, None


def rollout(s0, controls, engine, segment=None, theta=None):
    """States [T + 1, n_state, ld] of a T-step rollout, differentiable in s0 and controls
    [T, n_servo, ld], and in theta (the scene's parameters, `engine.theta()`) when given.
    segment: checkpoint every `segment` steps (None: keep every step's factor on the
    tape; the engine then needs T slots)."""
    if theta is not None:
        ref = engine.theta().to(dtype=theta.dtype)
        if theta.shape != ref.shape or not torch.allclose(theta.detach().cpu(), ref, rtol=1e-6, atol=0.0):
            raise ValueError("theta must hold the scene's own parameters (engine.theta())")
    return _Rollout.apply(s0, controls, theta, engine, segment)
