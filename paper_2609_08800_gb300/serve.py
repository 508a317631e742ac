"""Serving loop: continuous batching of rollout and optimisation requests.

A request asks for a rollout of `n` worlds of one scene over a horizon of `T` steps,
either forward only (the final states) or forward plus the adjoint sweep (the loss
gradient with respect to the initial states and to every step's servo targets).

Each scene kind has a `Pool`: one libostrich context of C world columns whose
states, gradient columns, tape (K slots per world), checkpoints (one state per
K-step segment of the longest horizon) and control tables stay resident on the
device.  The pool's size is set from the free HBM when it is created; a request is
admitted when its pool has `n` free columns (first fit in arrival order, with the
head of the queue reserving columns once it has waited `max_bypass` seconds, so
neither small nor large requests starve).  Columns are released when the request's
results have reached the host.

Every tick each pool issues, on its step stream, one `ostrich_step_list` over the
columns of all its requests that are stepping forward (no record, except that a
forward+adjoint request records its last segment, so that its backward sweep starts
without a re-run) or re-running a checkpointed segment (recording slot t - t0), and, on
its adjoint stream, one `ostrich_adjoint_list` over the columns of all requests sweeping
a segment backwards.
Requests at different steps of different horizons therefore share launches; the two
streams of a pool and the pools themselves run concurrently.  Tick t of the step
stream waits for tick t-1 of the adjoint stream and vice versa, which orders every
hand-over of a request between the two (final state -> loss gradient, segment
re-run -> its adjoints -> the previous segment's re-run).

A world's result depends only on its own inputs: each CTA steps one world, reads only
its own column and reduces in a fixed order, so a request's result is the same
whether it runs alone or among others (for a fixed threads-per-world setting).
"""
from __future__ import annotations

import heapq
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import scenes as S
from . import spline as SP
from .ostrich import Context

FWD, REC, ADJ, DONE = 0, 1, 2, 3


@dataclass
class Request:
    rid: int
    kind: str
    n: int
    T: int
    adjoint: bool
    arrival: float = 0.0
    seed: int = 0
    # inputs: initial states [n_state, n], servo targets [T, n_servo, n] (host, float64)
    s0: np.ndarray = None
    controls: np.ndarray = None
    # results (host tensors)
    final_state: torch.Tensor = None
    loss: torch.Tensor = None
    dstate0: torch.Tensor = None
    dcontrols: torch.Tensor = None
    # schedule bookkeeping
    cols: np.ndarray = None
    phase: int = FWD
    t: int = 0
    seg: int = 0
    admitted_at: float = 0.0
    done_at: float = 0.0
    _event: object = None
    _entered: bool = False
    _finish_pending: bool = False


def loss_grad(kind, state, nb):
    """Loss per world and its gradient with respect to the final state.  Box: final x
    position.  Robot / terrain: squared chassis distance to (3, 0) in the plane."""
    g = torch.zeros_like(state)
    if kind == "box":
        loss = state[0].clone()
        g[0] = 1.0
    else:
        loss = (state[0] - 3.0) ** 2 + state[1] ** 2
        g[0] = 2.0 * (state[0] - 3.0)
        g[1] = 2.0 * state[1]
    return loss, g


def scene_of(kind):
    if kind == "box":
        return S.box_drop_scene()
    if kind == "robot":
        return S.robot_box_scene()
    if kind == "terrain":
        return S.terrain_scene()
    raise ValueError(kind)


def request_inputs(kind, scene, n, T, seed, h):
    """Seeded initial states and servo targets of a request (box: initial velocity
    U[0, 1] m/s; robots: placements of the robot generators and 8-knot wheel splines
    uniform in [-5, 5] rad/s)."""
    rng = np.random.default_rng(seed)
    if kind == "box":
        s0 = np.concatenate([S.box_drop_state(scene, float(v)) for v in rng.uniform(0.0, 1.0, n)], axis=1)
        return s0, np.zeros((T, 0, n))
    if kind == "robot":
        s0 = S.robot_box_states(scene, n, seed=seed)
    else:
        s0 = S.terrain_states(scene, n, seed=seed)
    knots = S.spline_knots(n, n_wheels=scene.n_servos, n_knots=8, seed=seed + 1)
    controls = np.ascontiguousarray(np.einsum("tk,wjk->tjw", SP.basis(T, 8, h), knots))   # [T, n_servo, n]
    return s0, controls


def poisson_stream(rate, duration, seed, kinds=("box", "robot", "terrain"), max_worlds=512, horizon=(20, 200)):
    """Seeded request stream: Poisson arrivals of mean `rate` per second over
    `duration` seconds; worlds log-uniform in [1, max_worlds]; horizon uniform in
    `horizon`; scene uniform over `kinds`; half forward-only, half forward+adjoint."""
    rng = np.random.default_rng(seed)
    reqs, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        n = int(np.clip(np.floor(np.exp(rng.uniform(0.0, math.log(max_worlds + 1)))), 1, max_worlds))
        T = int(rng.integers(horizon[0], horizon[1] + 1))
        kind = kinds[int(rng.integers(len(kinds)))]
        reqs.append(Request(rid=len(reqs), kind=kind, n=n, T=T, adjoint=bool(rng.integers(2)), arrival=t,
                            seed=int(rng.integers(1 << 30))))
    return reqs


class _Ring:
    """Pinned host staging buffers reused every `depth` ticks."""

    def __init__(self, depth, size):
        self.bufs = [torch.empty(size, dtype=torch.int32, pin_memory=True) for _ in range(depth)]
        self.k = 0

    def next(self, n):
        b = self.bufs[self.k]
        self.k = (self.k + 1) % len(self.bufs)
        if b.numel() < n:
            raise RuntimeError("staging buffer too small")
        return b


class Pool:
    """Resident device state of one scene kind."""

    def __init__(self, kind, cfg, capacity, h=0.1, K=10, t_max=200, dtype="f32", threads=None, hbm_share=None):
        self.kind, self.h, self.K, self.t_max = kind, h, K, t_max
        self.scene = scene_of(kind)
        probe = Context(self.scene, cfg, 1, dtype=dtype, tape_slots=1)
        per_world = self._bytes_per_world(probe, K, t_max)
        probe.close()
        if hbm_share is not None:
            free, _ = torch.cuda.mem_get_info()
            capacity = max(1, min(capacity, int(free * hbm_share // per_world)))
        self.C = capacity
        self.bytes_per_world = per_world
        self.ctx = Context(self.scene, cfg, capacity, dtype=dtype, tape_slots=K, threads=threads)
        c, dt, dev = self.ctx, self.ctx.dtype, "cuda"
        ns, nsv = c.n_state, max(c.n_servo, 1)
        self.nb = self.scene.n_bodies
        self.S = torch.zeros(ns, capacity, dtype=dt, device=dev)
        self.G = torch.zeros(ns, capacity, dtype=dt, device=dev)
        self.ctl = torch.zeros(nsv, capacity, dtype=dt, device=dev)
        self.dctl = torch.zeros(nsv, capacity, dtype=dt, device=dev)
        self.CT = torch.zeros(t_max, nsv, capacity, dtype=dt, device=dev)       # servo targets
        self.DCT = torch.zeros(t_max, nsv, capacity, dtype=dt, device=dev)      # their gradients
        self.CK = torch.zeros((t_max + K - 1) // K, ns, capacity, dtype=dt, device=dev)   # checkpoints
        self.free = list(range(capacity))
        heapq.heapify(self.free)
        self.sa, self.sb = torch.cuda.Stream(), torch.cuda.Stream()
        self.ev_a = self.ev_b = None
        self.ring_a, self.ring_b = _Ring(4, 3 * capacity + 8), _Ring(4, 3 * capacity + 8)
        self.active = []

    @staticmethod
    def _bytes_per_world(ctx, K, t_max):
        es = 8 if ctx.dtype == torch.float64 else 4
        ns, nsv = ctx.n_state, max(ctx.n_servo, 1)
        tape = ctx.tape_bytes()                      # one slot of one world
        return K * tape + es * (2 * ns + 2 * nsv + 2 * t_max * nsv + ((t_max + K - 1) // K) * ns)

    def n_free(self):
        return len(self.free)

    def admit(self, r):
        r.cols = np.array(sorted(heapq.heappop(self.free) for _ in range(r.n)), dtype=np.int64)
        r.phase, r.t, r._entered = FWD, 0, False
        self.active.append(r)

    def release(self, r):
        for c in r.cols.tolist():
            heapq.heappush(self.free, c)


class Server:
    """Continuous-batching loop over a set of pools."""

    def __init__(self, pools, max_bypass=0.5, clock=time.perf_counter, fifo=False):
        """fifo=True serves one request at a time in arrival order (a queue without
        batching), the baseline continuous batching is measured against."""
        self.pools = {p.kind: p for p in pools}
        self.max_bypass = max_bypass
        self.fifo = fifo
        self.clock = clock
        self.queue = []
        self.inflight = []          # requests whose results are being copied out
        self.done = []
        self.tick = 0
        self.world_steps = 0

    # ---- admission -------------------------------------------------------------------
    def _admit(self, now):
        if self.fifo:
            if self.queue and not any(p.active for p in self.pools.values()):
                r = self.queue.pop(0)
                self._start(self.pools[r.kind], r, now)
            return
        blocked = set()
        keep = []
        for r in self.queue:
            p = self.pools[r.kind]
            if r.kind not in blocked and p.n_free() >= r.n:
                self._start(p, r, now)
            else:
                keep.append(r)
                if now - r.arrival > self.max_bypass:
                    blocked.add(r.kind)          # head-of-line reservation for a waiting request
        self.queue = keep

    def submit(self, r):
        p = self.pools.get(r.kind)
        if p is None:
            raise ValueError(f"no pool serves scene kind {r.kind!r}")
        if r.n > p.C or r.T > p.t_max:
            raise ValueError(f"request {r.rid}: {r.n} worlds x {r.T} steps exceeds the pool ({p.C} x {p.t_max})")
        self.queue.append(r)

    def _start(self, p, r, now):
        if r.s0 is None:
            r.s0, r.controls = request_inputs(r.kind, p.scene, r.n, r.T, r.seed, p.h)
        p.admit(r)
        r.admitted_at = now
        dt = p.ctx.dtype
        # inputs go up from pinned staging copies, asynchronously on the step stream
        # (allocated there; the tensors stay referenced by the request until it is done)
        r._pinned = [torch.from_numpy(r.cols).pin_memory(),
                     torch.from_numpy(np.ascontiguousarray(r.s0)).to(dt).pin_memory(),
                     torch.from_numpy(np.ascontiguousarray(r.controls)).to(dt).pin_memory()]
        with torch.cuda.stream(p.sa):
            cols = r._pinned[0].to("cuda", non_blocking=True)
            p.S[:, cols] = r._pinned[1].to("cuda", non_blocking=True)
            if r.controls.shape[1]:
                p.CT[:r.T, :r.controls.shape[1], :][:, :, cols] = r._pinned[2].to("cuda", non_blocking=True)
        r._cols_dev = cols

    # ---- one tick ----------------------------------------------------------------------
    def _tick_pool(self, p):
        K = p.K
        step_w, step_s, step_t, adj_w, adj_s, adj_t = [], [], [], [], [], []
        saves, restores, to_bwd, finish_a, finish_b = [], [], [], [], []
        for r in p.active:
            if r._finish_pending:
                continue
            if r.phase == FWD and r.t < r.T:
                # a forward+adjoint request checkpoints every segment start but the last
                # and records the last segment's steps (slot t - t_last)
                t_last = ((r.T - 1) // K) * K
                rec = r.adjoint and r.t >= t_last
                if r.adjoint and r.t % K == 0 and not rec:
                    saves.append(r)
                step_w.append(r.cols); step_s.append(np.full(r.n, r.t - t_last if rec else -1))
                step_t.append(np.full(r.n, r.t))
            elif r.phase == REC:
                t0 = r.seg * K
                if r.t == t0:
                    restores.append(r)
                step_w.append(r.cols); step_s.append(np.full(r.n, r.t - t0)); step_t.append(np.full(r.n, r.t))
            elif r.phase == ADJ:
                t0 = r.seg * K
                adj_w.append(r.cols); adj_s.append(np.full(r.n, r.t - t0)); adj_t.append(np.full(r.n, r.t))
        # ---- step stream
        with torch.cuda.stream(p.sa):
            if p.ev_b is not None:
                p.sa.wait_event(p.ev_b)
            for r in saves:
                p.CK[r.t // K][:, r._cols_dev] = p.S[:, r._cols_dev]
            for r in restores:
                p.S[:, r._cols_dev] = p.CK[r.seg][:, r._cols_dev]
            if step_w:
                lw, ls, lt = self._stage(p.ring_a, step_w, step_s, step_t)
                if p.ctx.n_servo:
                    p.ctl[:, lw.long()] = p.CT[lt.long(), :, lw.long()].T
                p.ctx.ostrich_step_list(p.S, p.ctl, p.h, p.S, lw, ls)
            ev_a = torch.cuda.Event()
            ev_a.record(p.sa)
        # ---- adjoint stream
        with torch.cuda.stream(p.sb):
            if p.ev_a is not None:
                p.sb.wait_event(p.ev_a)
            for r in p.active:
                if r.phase == FWD and r.t == r.T and not r._finish_pending and r.adjoint:
                    to_bwd.append(r)
            for r in to_bwd:
                fs = p.S[:, r._cols_dev]
                r._loss, g = loss_grad(r.kind, fs, p.nb)
                r._final = fs
                p.G[:, r._cols_dev] = g
            if adj_w:
                lw, ls, lt = self._stage(p.ring_b, adj_w, adj_s, adj_t)
                p.ctx.ostrich_adjoint_list(p.G, p.h, p.G, lw, ls, p.dctl if p.ctx.n_servo else None)
                if p.ctx.n_servo:
                    p.DCT[lt.long(), :, lw.long()] = p.dctl[:, lw.long()].T
            ev_b = torch.cuda.Event()
            ev_b.record(p.sb)
        # ---- advance the schedules (host)
        for r in p.active:
            if r._finish_pending:
                continue
            if r.phase == FWD:
                if r.t < r.T:
                    r.t += 1
                    self.world_steps += r.n
                    if r.t == r.T and not r.adjoint:
                        finish_a.append(r)
                elif r in to_bwd:
                    # the last segment is on the tape: its adjoint sweep starts at once
                    r.phase, r.seg = ADJ, (r.T - 1) // K
                    r.t = r.T - 1
            elif r.phase == REC:
                r.t += 1
                if r.t == min(r.T, (r.seg + 1) * K):
                    r.phase, r.t = ADJ, r.t - 1
            elif r.phase == ADJ:
                if r.t == r.seg * K:
                    if r.seg == 0:
                        finish_b.append(r)
                    else:
                        r.seg -= 1
                        r.phase, r.t = REC, r.seg * K
                else:
                    r.t -= 1
        # ---- results of finished requests
        for r in finish_a:
            with torch.cuda.stream(p.sa):
                fs = p.S[:, r._cols_dev]
                r.loss = torch.empty(r.n, dtype=fs.dtype, pin_memory=True)
                r.final_state = torch.empty(fs.shape, dtype=fs.dtype, pin_memory=True)
                loss, _ = loss_grad(r.kind, fs, p.nb)
                r.loss.copy_(loss, non_blocking=True)
                r.final_state.copy_(fs, non_blocking=True)
                r._event = torch.cuda.Event()
                r._event.record(p.sa)
            r._finish_pending = True
        for r in finish_b:
            with torch.cuda.stream(p.sb):
                c = r._cols_dev
                r.loss = torch.empty(r.n, dtype=p.S.dtype, pin_memory=True)
                r.final_state = torch.empty(p.S.shape[0], r.n, dtype=p.S.dtype, pin_memory=True)
                r.dstate0 = torch.empty(p.S.shape[0], r.n, dtype=p.S.dtype, pin_memory=True)
                r.loss.copy_(r._loss, non_blocking=True)
                r.final_state.copy_(r._final, non_blocking=True)
                r.dstate0.copy_(p.G[:, c], non_blocking=True)
                if p.ctx.n_servo:
                    r.dcontrols = torch.empty(r.T, p.ctx.n_servo, r.n, dtype=p.S.dtype, pin_memory=True)
                    r.dcontrols.copy_(p.DCT[:r.T, :p.ctx.n_servo][:, :, c], non_blocking=True)
                r._event = torch.cuda.Event()
                r._event.record(p.sb)
            r._finish_pending = True
        p.ev_a, p.ev_b = ev_a, ev_b
        return ev_a, ev_b

    @staticmethod
    def _stage(ring, ws, ss, ts):
        w = np.concatenate(ws)
        n = w.size
        buf = ring.next(3 * n)
        host = buf[:3 * n].numpy().reshape(3, n)
        host[0] = w
        host[1] = np.concatenate(ss)
        host[2] = np.concatenate(ts)
        dev = buf[:3 * n].to("cuda", non_blocking=True).view(3, n)
        return dev[0], dev[1], dev[2]

    def _collect(self, now):
        for p in self.pools.values():
            keep = []
            for r in p.active:
                if r._finish_pending and r._event.query():
                    r.done_at = self.clock()
                    r.phase = DONE
                    p.release(r)
                    self.done.append(r)
                else:
                    keep.append(r)
            p.active = keep

    def busy(self):
        return bool(self.queue) or any(p.active for p in self.pools.values())

    def run(self, requests, t0=None, max_inflight_ticks=2, deadline=None):
        """Serve `requests` (sorted by arrival time, seconds from t0) until all are done, or
        until `deadline` seconds after t0: requests not finished by then (queued, or in
        flight, whose launches are drained but whose results are dropped) are left in
        `self.unfinished`."""
        pending = sorted(requests, key=lambda r: r.arrival)
        t0 = self.clock() if t0 is None else t0
        i = 0
        history = []
        self.unfinished = []
        while i < len(pending) or self.busy():
            now = self.clock() - t0
            if deadline is not None and now >= deadline:
                self.unfinished = list(self.queue) + [r for p in self.pools.values() for r in p.active]
                self.unfinished += pending[i:]
                break
            while i < len(pending) and pending[i].arrival <= now:
                self.submit(pending[i])
                i += 1
            self._admit(now)
            if not any(p.active for p in self.pools.values()):
                if i < len(pending):
                    time.sleep(max(0.0, pending[i].arrival - (self.clock() - t0)))
                continue
            evs = []
            for p in self.pools.values():
                if p.active:
                    evs.extend(self._tick_pool(p))
            history.append(evs)
            if len(history) > max_inflight_ticks:
                for e in history.pop(0):
                    e.synchronize()
            self._collect(now)
            self.tick += 1
        torch.cuda.synchronize()
        self._collect(self.clock() - t0)
        for r in self.done:
            r.latency = r.done_at - t0 - r.arrival
        return self.done


def summarize(done, wall, unfinished=(), cutoff=None):
    """Latency percentiles of the finished requests and world-steps/s.  With a cutoff, the
    requests left unfinished get the censored latency cutoff - arrival (a lower bound on
    their true latency, for those that had arrived), and `censored_p50_s` /
    `censored_p99_s` over all arrived requests are lower bounds on the stream's p50/p99."""
    lat = np.array([r.latency for r in done]) if done else np.zeros(1)
    ws = sum(r.n * r.T for r in done)
    out = {"requests": len(done), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
           "world_steps": ws, "world_steps_per_s": ws / wall if wall > 0 else 0.0}
    if cutoff is not None:
        arrived = [r for r in unfinished if r.arrival <= cutoff]
        cens = np.concatenate([lat if done else np.zeros(0), np.array([cutoff - r.arrival for r in arrived])])
        out.update({"cutoff_s": cutoff, "unfinished": len(arrived), "not_arrived": len(unfinished) - len(arrived),
                    "censored_p50_s": float(np.percentile(cens, 50)) if cens.size else 0.0,
                    "censored_p99_s": float(np.percentile(cens, 99)) if cens.size else 0.0})
    return out


class PlainServer:
    """The plain form of the same service: one request at a time in arrival order, and
    within a request one world per launch (W = 1 contexts over the pool's columns), the
    same steps, segment checkpoints and adjoint sweeps as the batched server.  It is the
    baseline the continuous-batching latency is compared against."""

    def __init__(self, pools, clock=time.perf_counter):
        self.pools = {p.kind: p for p in pools}
        self.clock = clock
        self.done, self.unfinished = [], []

    def _serve(self, r):
        p = self.pools[r.kind]
        if r.s0 is None:
            r.s0, r.controls = request_inputs(r.kind, p.scene, r.n, r.T, r.seed, p.h)
        dt, K, n = p.ctx.dtype, p.K, r.n
        # one world per launch: a W = 1 context whose arrays are strided by the request's n
        ctx = Context(p.scene, p.ctx.cfg, 1, dtype="f64" if dt == torch.float64 else "f32", tape_slots=K, ld=n,
                      threads=getattr(p.ctx, "threads", None))
        S0 = torch.from_numpy(np.ascontiguousarray(r.s0)).to(dtype=dt).pin_memory().to("cuda", non_blocking=True)
        nsv = p.ctx.n_servo
        CT = (torch.from_numpy(np.ascontiguousarray(r.controls)).to(dtype=dt).pin_memory().to("cuda", non_blocking=True)
              if nsv else torch.zeros(r.T, 1, n, dtype=dt, device="cuda"))
        n_seg = (r.T + K - 1) // K
        ns = S0.shape[0]
        st = torch.empty(2, ns, n, dtype=dt, device="cuda")
        st[0] = S0
        ck = torch.empty(n_seg, ns, n, dtype=dt, device="cuda")
        g = torch.empty(2, ns, n, dtype=dt, device="cuda")
        dct = torch.zeros(r.T, max(nsv, 1), n, dtype=dt, device="cuda")
        fin = torch.empty(ns, n, dtype=dt, device="cuda")
        t_last = (n_seg - 1) * K
        for w in range(n):
            cur = 0
            for t in range(r.T):
                rec = r.adjoint and t >= t_last
                if r.adjoint and t % K == 0 and not rec:
                    ck[t // K, :, w] = st[cur, :, w]
                ctx.ostrich_step(_Column(st[cur], w), _Column(CT[t], w), p.h, _Column(st[1 - cur], w),
                                 tape_slot=t - t_last if rec else -1)
                cur = 1 - cur
            fin[:, w] = st[cur, :, w]
            if not r.adjoint:
                continue
            _, gw = loss_grad(r.kind, st[cur, :, w:w + 1], p.nb)
            g[0, :, w] = gw[:, 0]
            gc = 0
            for k in reversed(range(n_seg)):
                t0, t1 = k * K, min(r.T, (k + 1) * K)
                if k < n_seg - 1:                # the last segment was recorded by the forward
                    st[0, :, w] = ck[k, :, w]
                    cur = 0
                    for t in range(t0, t1):
                        ctx.ostrich_step(_Column(st[cur], w), _Column(CT[t], w), p.h, _Column(st[1 - cur], w),
                                         tape_slot=t - t0)
                        cur = 1 - cur
                for t in reversed(range(t0, t1)):
                    ctx.ostrich_adjoint(t - t0, _Column(g[gc], w), p.h, _Column(g[1 - gc], w),
                                        _Column(dct[t], w) if nsv else None)
                    gc = 1 - gc
            st[0, :, w] = g[gc, :, w]           # dL/ds0 of world w (st[0] is free again)
        loss, _ = loss_grad(r.kind, fin, p.nb)
        r.loss, r.final_state = loss.cpu(), fin.cpu()
        if r.adjoint:
            r.dstate0 = st[0].cpu()
            r.dcontrols = dct[:, :nsv].cpu() if nsv else None
        ctx.close()

    def run(self, requests, t0=None, deadline=None):
        pending = sorted(requests, key=lambda r: r.arrival)
        t0 = self.clock() if t0 is None else t0
        self.done, self.unfinished = [], []
        for i, r in enumerate(pending):
            now = self.clock() - t0
            if deadline is not None and now >= deadline:
                self.unfinished = pending[i:]
                break
            if r.arrival > now:
                time.sleep(r.arrival - now)
            self._serve(r)
            torch.cuda.synchronize()
            r.done_at = self.clock()
            r.latency = r.done_at - t0 - r.arrival
            self.done.append(r)
        return self.done


class _Column:
    """Column c of a dense [rows, C] device tensor: the address a W = 1 context with
    ld = C reads and writes (element c, then every C-th element)."""
    is_cuda = True

    def __init__(self, t, c):
        assert t.is_contiguous()
        self._p = t.data_ptr() + c * t.element_size()

    def data_ptr(self):
        return self._p

    def is_contiguous(self):
        return True
