"""Benchmark: forward + adjoint world-steps/s of the Ostrich per-step solve on GB300.

Headline workload (one bench step = one optimisation iteration): the wheeled robot
over a box obstacle, 8192 worlds per GPU, FP32, 8-knot wheel-velocity splines per
world, a 100-step horizon (10 s at h = 0.1) rolled out through the autograd.Function
with checkpoints every 10 steps, the loss gradient swept back by the IFT adjoint (the
forward records the last 10-step segment into the tape, the backward recomputes each
earlier segment into the tape first), and an Adam update of
the knots (lr 0.3).  `value` counts W x T forward+adjoint world-steps per iteration
over all ranks (replicas: each GPU runs its own worlds); the recompute is counted as
cost, not as world-steps.  Inputs are resident in HBM when the timed region starts.

Prints one JSON line.  Extra keys:
  e2e            the same metric through the public API: every iteration copies its
                 initial states up from pinned host memory and reads the losses and the
                 updated knots back, inside the timed region
  chunk          one 10-step chunk (10 forward steps recording the tape, 10 adjoints)
                 repeated from the same states: per-kernel times, Newton histogram
  roofline       ALU roofline of the step kernel (algorithmic flops / event time) in the
                 chunk leg, against a measured FFMA peak
  plain_form     the same kernels launched once per world per step (W = 1)
  serving        the Poisson request stream: continuous batching, FIFO queue, plain form
  cpu_baseline   the FP64 oracle on the host cores, on a bounded sample
`--impl reference` times the FP64 oracle instead (the reference arm): each step one Adam
iteration of the same optimisation workload on a sample of worlds, split over the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2609_08800_gb300 import scenes as S  # noqa: E402
from paper_2609_08800_gb300 import spline as SP  # noqa: E402

METRIC = "fwd+adjoint world-steps/s @8192 worlds"
UNIT = "world-steps/s"
H = 0.1
CHUNK = 10
OPT_T = 100      # horizon of the optimisation workload (10 s at h = 0.1)
CHUNK_WARMUP, CHUNK_TIMED = 3, 5   # chunk leg: warm-up and timed chunks
FP32_TOL = 1e-4      # m/s: the FP32 residual floor of this scene (FP32-rounded exact states sit near 1e-5)
SM_COUNT_GB300 = 152
FP32_LANES_PER_SM = 128
L2_BYTES = 129 * 2 ** 20


# Refinement sweeps per Schur solve of the forward step kernel: none (the Newton
# iteration corrects an inexact step itself; only the adjoint's single solve is refined).
FORWARD_REFINE_SWEEPS = 0


def world_flops(iters, rows, groups, sep, refine=FORWARD_REFINE_SWEEPS, trials_per_iter=1):
    """Algorithmic FP32 flops of one world-step of the forward kernel (structured count).

    iters: Newton iterations run; rows: active rows m; groups: contact rows per body
    group p_g; sep: separator rows s.  Per evaluation 250 m (residual, Jacobian,
    dynamics); per assembly: group blocks 6 p(p+1), coupling 72 p, separator 12 s(s+1);
    per factorisation: sum p^3/3 + 6 p^2 + 36 p, plus s^3/3; per solve 2 (sum p^2 + s^2)
    + 24 sum p, plus 48 m per refinement product (the forward kernel runs none)."""
    m = rows
    ev = 250.0 * m
    asm = sum(6.0 * p * (p + 1) + 72.0 * p for p in groups) + 12.0 * sep * (sep + 1)
    fac = sum(p ** 3 / 3.0 + 6.0 * p * p + 36.0 * p for p in groups) + sep ** 3 / 3.0
    sol = 2.0 * (sum(p * p for p in groups) + sep * sep) + 24.0 * sum(groups)
    per_iter = asm + fac + (1 + refine) * sol + refine * 48.0 * m + trials_per_iter * ev
    return iters * per_iter + 2 * ev + asm + fac     # warm-start eval, final eval, taped factor


def world_bytes(scene, rows, tape_record_bytes, elem=4, persistent=True):
    """Algorithmic HBM bytes of one world-step of the forward kernel: the inputs it reads
    (q-, u-, the warm-start multipliers of its active rows, the servo targets), the
    outputs it writes (the whole next state, impulses, contact ids, status and
    iteration words), its tape record, and the schedule's per-world words."""
    nb = scene.n_bodies
    reads = (13 * nb + rows + scene.n_servos) * elem
    writes = (scene.n_state + scene.m_max) * elem + 4 * (scene.n_slots + 2)
    sched = 12 if persistent else 0
    return reads + writes + tape_record_bytes + sched


def sample_clocks_start(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except Exception:
        return None, None


def sample_clocks_stop(handle, path, gpu_index):
    p, f = handle
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    f.close()
    sms, maxs, reasons = [], [], set()
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or parts[0] != str(gpu_index):
            continue
        try:
            sms.append(float(parts[1])); maxs.append(float(parts[2]))
        except ValueError:
            continue
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for n, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sms:
        return None
    return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxs), "reasons": sorted(reasons), "samples": len(sms)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_inputs(n_worlds, seed=0):
    scene = S.robot_box_scene()
    states = S.robot_box_states(scene, n_worlds, seed=seed)
    knots = S.spline_knots(n_worlds, n_wheels=4, n_knots=8, seed=seed)
    T = 100
    B = SP.basis(T, 8, H)                        # [T, K] natural cubic spline, knots over [0, T h]
    controls = np.ascontiguousarray(np.einsum("tk,wjk->tjw", B, knots))   # [T, 4, W], world index fastest
    # cotangent of the chunk's last state: d/ds of |p_xy - (3, 0)|^2 of the chassis
    g = np.zeros((scene.n_state, n_worlds))
    g[0] = 2.0 * (states[0] - 3.0)
    g[1] = 2.0 * states[1]
    return scene, states, controls[:CHUNK].astype(np.float32), g


class Chunk:
    """Forward CHUNK steps recording the tape, then CHUNK adjoint steps, on one stream."""

    def __init__(self, ctx, torch, n_worlds):
        self.ctx, self.torch = ctx, torch
        dev = "cuda"
        ns, W = ctx.n_state, ctx.ld
        f32 = torch.float32
        self.states = [torch.empty(ns, W, dtype=f32, device=dev) for _ in range(CHUNK + 1)]
        self.imp = torch.empty(ctx.m_max, W, dtype=f32, device=dev)
        self.ids = torch.empty(ctx.n_slots, W, dtype=torch.int32, device=dev)
        self.status = torch.empty(W, dtype=torch.int32, device=dev)
        self.iters = [torch.empty(W, dtype=torch.int32, device=dev) for _ in range(CHUNK)]
        self.ids_all = [torch.empty(ctx.n_slots, W, dtype=torch.int32, device=dev) for _ in range(CHUNK)]
        self.g = [torch.empty(ns, W, dtype=f32, device=dev) for _ in range(CHUNK + 1)]
        self.dctl = torch.empty(CHUNK, ctx.n_servo, W, dtype=f32, device=dev)

    def run(self, s0, controls, gT, ev_step=None, ev_adj=None, record_ids=False):
        ctx = self.ctx
        self.states[0].copy_(s0)
        for t in range(CHUNK):
            if ev_step is not None:
                ev_step[t][0].record()
            ctx.ostrich_step(self.states[t], controls[t], H, self.states[t + 1], self.imp,
                             self.ids_all[t] if record_ids else self.ids, self.status, self.iters[t], tape_slot=t)
            if ev_step is not None:
                ev_step[t][1].record()
        self.g[CHUNK].copy_(gT)
        for t in reversed(range(CHUNK)):
            if ev_adj is not None:
                ev_adj[t][0].record()
            ctx.ostrich_adjoint(t, self.g[t + 1], H, self.g[t], self.dctl[t])
            if ev_adj is not None:
                ev_adj[t][1].record()


def run_ours(args, rank, world_size, local_rank):
    import torch
    from paper_2609_08800_gb300.ostrich import Context
    torch.cuda.set_device(local_rank)
    dev = "cuda"
    W = args.worlds
    scene, states, controls, g = make_inputs(W, seed=rank)
    cfg = S.SolverConfig(tol=FP32_TOL)
    ctx = Context(scene, cfg, W, dtype="f32", tape_slots=CHUNK, threads=args.threads)
    threads = args.threads
    if threads is None:
        from paper_2609_08800_gb300 import tune
        threads = tune.apply(ctx) or 64
        ctx.set_threads(threads)
    s0 = torch.tensor(states, dtype=torch.float32, device=dev)
    ctl = torch.tensor(controls, dtype=torch.float32, device=dev)
    gT = torch.tensor(g, dtype=torch.float32, device=dev)
    chunk = Chunk(ctx, torch, W)
    for _ in range(CHUNK_WARMUP):
        chunk.run(s0, ctl, gT, record_ids=True)
    torch.cuda.synchronize()
    dist_barrier()
    # live per-launch timing of the two kernels over the timed region
    n_chunks = CHUNK_TIMED
    evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(CHUNK)] for _ in range(n_chunks)]
    eva = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(CHUNK)] for _ in range(n_chunks)]
    clk_path = os.path.join(tempfile.gettempdir(), f"ostrich_clocks_rank{rank}_{os.getpid()}.csv")
    clk = sample_clocks_start(clk_path)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record()
    for k in range(n_chunks):
        chunk.run(s0, ctl, gT, evs[k], eva[k])
    stop.record()
    torch.cuda.synchronize()
    clocks = sample_clocks_stop(clk, clk_path, local_rank)
    ms = start.elapsed_time(stop) / n_chunks
    from paper_2609_08800_gb300.ostrich import probe_ffma
    peak_ffma, probe_ms = probe_ffma()
    ms = dist_max(ms)
    step_ms = [e[0].elapsed_time(e[1]) for k in range(n_chunks) for e in evs[k]]
    adj_ms = [e[0].elapsed_time(e[1]) for k in range(n_chunks) for e in eva[k]]
    # algorithmic flops of the step launches (from the warm-up run: same inputs, same work)
    iters = np.stack([t.cpu().numpy() for t in chunk.iters])           # [CHUNK, W]
    ids = np.stack([t.cpu().numpy() for t in chunk.ids_all])           # [CHUNK, slots, W]
    n_iter = iters & 0xFFFF
    n_rows = iters >> 16
    sep = 5 * len(scene.joints) + scene.n_servos
    flops = 0.0
    tape_rec = ctx.tape_bytes() / ctx.n_worlds
    sched_on = getattr(ctx, "schedule", 0) == 1
    traffic = float(sum(world_bytes(scene, int(r), tape_rec, persistent=sched_on) for r in n_rows.ravel())) / CHUNK
    for t in range(CHUNK):
        for w in range(W):
            groups = []
            for b in range(scene.n_bodies):
                n = scene.slots_of_body(b)
                if n == 0:
                    continue
                base = sum(scene.slots_of_body(bb) for bb in range(b))
                groups.append(3 * int((ids[t, base:base + n, w] >= 0).sum()))
            flops += world_flops(int(n_iter[t, w]), int(n_rows[t, w]), groups, sep)
    flops_per_launch = flops / CHUNK
    avg_step_ms = statistics.mean(step_ms)
    achieved = flops_per_launch / (avg_step_ms * 1e-3) / 1e12
    sm_mhz = (clocks or {}).get("sm_mhz") or measured_peaks().get("sm_max_mhz", 2070.0)
    peak_derived = SM_COUNT_GB300 * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    chunk_value = W * CHUNK * world_size / (ms * 1e-3)
    traj_b, seg_b = (OPT_T + 1) * ctx.n_state * W * 4, CHUNK * ctx.tape_bytes()     # tape_bytes: one slot
    l2_note = (f"trajectory {traj_b / 1e9:.2f} GB and tape of one segment {seg_b / 1e9:.2f} GB per iteration "
               + ("> 129 MB L2 (no flush needed)" if min(traj_b, seg_b) > L2_BYTES else
                  "(at this world count not all beyond the 129 MB L2: not a bench-sized run)"))
    opt = run_optimisation(args, torch, rank, world_size)
    out = {
        "metric": METRIC, "value": opt["value"], "unit": UNIT, "n_gpus": world_size, "steps": opt["iterations"],
        "warmup": args.warmup, "ms_per_step": opt["ms_per_iteration"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(opt_config(W), newton_budget=cfg.budget, threads_per_world=opt["threads_per_world"],
                       parallelism=f"replicas{world_size}",
                       l2=l2_note),
        "gpu_launches": opt["gpu_launches_per_iteration"] * opt["iterations"],
        "e2e": opt["e2e"],
        "optimisation": {k: opt[k] for k in ("loss_first_warmup", "loss_first_timed", "loss_last_timed",
                                             "last_iteration_ms", "iterations")},
        "chunk": {"workload": f"robot_over_box_{W}_worlds_fp32_fwd_adj_chunk10 (every chunk restarts from the same "
                              "states: steps 1-10 of the horizon, tape recorded in the forward, no recompute)",
                  "value": chunk_value, "unit": UNIT, "ms_per_chunk": ms, "timed_chunks": n_chunks,
                  "warmup_chunks": CHUNK_WARMUP, "schedule": getattr(ctx, "schedule", 0)},
        "kernels": {"step_ms_avg": avg_step_ms, "adjoint_ms_avg": statistics.mean(adj_ms),
                    "newton_iters_mean": float(n_iter.mean()), "active_rows_mean": float(n_rows.mean()),
                    "newton_iters_hist": np.bincount(n_iter.ravel(), minlength=cfg.budget + 1).tolist()},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_ffma, "unit": "TFLOP/s",
                     "frac": achieved / peak_ffma,
                     "traffic": traffic,
                     "traffic_source": "algorithmic bytes of one step launch: per world q-, u-, warm-start "
                                       "multipliers of the active rows and servo targets read; next state, "
                                       "impulses, ids, status and iteration words, the tape record and the "
                                       "schedule words written (the DRAM bytes ncu measures for the same "
                                       "launch are in profiles/)",
                     "hbm_gbs_achieved": traffic / (avg_step_ms * 1e-3) / 1e9,
                     "timed_region": "the chunk leg (step launches timed one by one with CUDA events)",
                     "peak_source": f"measured: FFMA-only probe kernel (ostrich_probe_ffma), {probe_ms:.1f} ms "
                                    f"per launch, run beside the timed region",
                     "peak_derived": peak_derived,
                     "peak_derived_source": f"152 SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz "
                                            "(median SM clock sampled in the timed region)",
                     "kernel": "step_kernel<float>", "flops_per_launch": flops_per_launch},
    }
    if opt["clocks"]:
        out["clocks"] = opt["clocks"]
    if clocks:
        out["chunk"]["clocks"] = clocks
    if rank == 0 and not args.skip_extras:
        out["adjoint_modes"] = run_param_grads(ctx, chunk, torch)
        out["chunk"]["e2e"] = run_e2e(args, ctx, chunk, states, controls, g, torch)
        out["plain_form"] = run_plain(args, scene, cfg, states, controls, g, torch)
        out["cpu_baseline"] = run_cpu_baseline(args)
        if args.terrain_worlds > 0:
            out["terrain"] = run_terrain(args, torch)
        if args.linear_solvers:
            out["linear_solvers"] = run_linear_solvers(args, torch)
        if args.serve_seconds > 0:
            out["serving"] = run_serving(args, torch)
    ctx.close()
    return out


def run_optimisation(args, torch, rank, world_size):
    """The optimisation workload: the robot over the box obstacle, args.worlds worlds per GPU, FP32,
    8-knot wheel-velocity splines per world (seeded), horizon T = 100 at h = 0.1, rollout
    through the autograd.Function with checkpoints every 10 steps (the forward records the
    last segment into the tape; the backward sweeps it from there and recomputes each
    earlier segment into the tape before sweeping the adjoint back through it), loss =
    squared chassis distance to (3, 0) summed over the worlds, Adam on the knots with lr
    0.3 (Sec. IV-B).  A bench step is one optimisation iteration: W x T forward steps,
    W x (T - 10) recomputed steps and W x T adjoint steps; world-steps count W x T per
    iteration."""
    from paper_2609_08800_gb300 import tune
    from paper_2609_08800_gb300.autograd import CudaEngine, rollout
    W, T = args.worlds, OPT_T
    scene = S.robot_box_scene()
    states = S.robot_box_states(scene, W, seed=rank)
    knots0 = S.spline_knots(W, n_wheels=4, n_knots=8, seed=rank)
    cfg = S.SolverConfig(tol=FP32_TOL)
    eng = CudaEngine(scene, cfg, W, H, slots=CHUNK, dtype="f32")
    threads = tune.apply(eng.ctx) or 64
    B = torch.tensor(SP.basis(T, 8, H), dtype=torch.float32, device="cuda")          # [T, K]
    s0 = torch.tensor(states, dtype=torch.float32, device="cuda")
    knots = torch.tensor(knots0, dtype=torch.float32, device="cuda").requires_grad_(True)
    opt = torch.optim.Adam([knots], lr=0.3)

    phase_ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def iteration(s_init, mark=False):
        opt.zero_grad(set_to_none=True)
        controls = torch.einsum("tk,wjk->tjw", B, knots).contiguous()                  # [T, 4, W]
        if mark:
            phase_ev[0].record()
        traj = rollout(s_init, controls, eng, segment=CHUNK)
        sT = traj[T]
        loss_w = (sT[0] - 3.0) ** 2 + sT[1] ** 2
        if mark:
            phase_ev[1].record()
        # worlds whose rollout diverged (non-finite state) contribute no gradient
        torch.where(torch.isfinite(loss_w), loss_w, torch.zeros_like(loss_w)).sum().backward()
        if mark:
            phase_ev[2].record()
        # a world whose rollout diverged keeps its knots (its adjoint ran through
        # non-finite states)
        torch.nan_to_num_(knots.grad, nan=0.0, posinf=0.0, neginf=0.0)
        opt.step()
        return loss_w.detach()

    def loss_stats(lw):
        fin = torch.isfinite(lw)
        return {"mean_finite": float(lw[fin].mean()), "non_finite_worlds": int((~fin).sum())}

    first = None
    for _ in range(args.warmup):
        lw = iteration(s0)
        first = lw if first is None else first
    torch.cuda.synchronize()
    dist_barrier()
    clk_path = os.path.join(tempfile.gettempdir(), f"ostrich_opt_clocks_rank{rank}_{os.getpid()}.csv")
    clk = sample_clocks_start(clk_path)
    K = max(1, args.steps)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    losses = []
    for k in range(K):
        losses.append(iteration(s0, mark=(k == K - 1)))
    b.record()
    torch.cuda.synchronize()
    dist_barrier()
    clocks = sample_clocks_stop(clk, clk_path, int(os.environ.get("LOCAL_RANK", "0")))
    ms = dist_max(a.elapsed_time(b) / K)
    fwd_ms, bwd_ms = phase_ev[0].elapsed_time(phase_ev[1]), phase_ev[1].elapsed_time(phase_ev[2])
    # end to end through the public API: each iteration copies its initial states up from
    # pinned host memory and reads the per-world losses and the updated knots back
    hs0 = torch.tensor(states, dtype=torch.float32).pin_memory()
    hloss = torch.empty(W, dtype=torch.float32).pin_memory()
    hknots = torch.empty(knots.shape, dtype=torch.float32).pin_memory()
    ds0 = torch.empty_like(s0)
    n_e2e = min(K, 5)
    torch.cuda.synchronize()
    a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a2.record()
    for _ in range(n_e2e):
        ds0.copy_(hs0, non_blocking=True)
        lw = iteration(ds0)
        hloss.copy_(lw, non_blocking=True)
        hknots.copy_(knots.detach(), non_blocking=True)
    b2.record()
    torch.cuda.synchronize()
    ms_e2e = dist_max(a2.elapsed_time(b2) / n_e2e)
    eng.close()
    ws = W * T * world_size
    return {"value": ws / (ms * 1e-3), "ms_per_iteration": ms, "iterations": K, "warmup": args.warmup,
            "threads_per_world": threads, "clocks": clocks,
            "loss_first_warmup": None if first is None else loss_stats(first),
            "loss_first_timed": loss_stats(losses[0]), "loss_last_timed": loss_stats(losses[-1]),
            "last_iteration_ms": {"forward_rollout": fwd_ms, "backward_recompute_and_adjoint": bwd_ms},
            # per step launch one heaviest-first ordering launch (persistent schedule); forward T steps, the
            # recomputed segments T - CHUNK steps, T adjoints
            "gpu_launches_per_iteration": 2 * T + 2 * (T - CHUNK) + T,
            "e2e": {"value": ws / (ms_e2e * 1e-3), "unit": UNIT, "ms_per_iteration": ms_e2e, "iterations": n_e2e,
                    "h2d_bytes_per_step": hs0.numel() * 4,
                    "d2h_bytes_per_step": (hloss.numel() + hknots.numel()) * 4}}


def run_param_grads(ctx, chunk, torch, reps=5):
    """The adjoint launches of the chunk's ten recorded steps (slots 0-9, 8192 worlds) in
    the paper's mode, in the paper's mode with the physical-parameter gradients (servo
    gains, body masses, inertias, mu; Eq. (17) with xi = theta) and in the exact IFT mode,
    timed with CUDA events; the exact mode's GMRES iterations per world."""
    from paper_2609_08800_gb300.ostrich import ADJ_EXACT, ADJ_PAPER
    W = ctx.ld
    dev = "cuda"
    ds = torch.empty(ctx.n_state, W, dtype=torch.float32, device=dev)
    du = torch.empty(ctx.n_servo, W, dtype=torch.float32, device=dev)
    dkp = torch.empty(ctx.n_servo, W, dtype=torch.float32, device=dev)
    dm = torch.empty(ctx.nb, W, dtype=torch.float32, device=dev)
    di = torch.empty(3 * ctx.nb, W, dtype=torch.float32, device=dev)
    dmu = torch.empty(W, dtype=torch.float32, device=dev)
    kry = torch.zeros(CHUNK, W, dtype=torch.int32, device=dev)

    def timed(fn):
        for t in range(CHUNK):
            fn(t)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            for t in range(CHUNK):
                fn(t)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / (reps * CHUNK)

    plain = timed(lambda t: ctx.ostrich_adjoint(t, chunk.g[t + 1], H, ds, du))
    params = timed(lambda t: ctx.ostrich_adjoint_params(t, chunk.g[t + 1], H, ds, du, dkp, dm, di, dmu))

    def exact(t):
        ctx.set_adjoint_mode(ADJ_EXACT, kry[t])
        ctx.ostrich_adjoint(t, chunk.g[t + 1], H, ds, du)

    ex_ms = timed(exact)
    ctx.set_adjoint_mode(ADJ_PAPER)
    k = kry.cpu().numpy()
    its = k & 0xFFFF
    return {"worlds": W, "launches": f"the {CHUNK} recorded steps of the chunk, {reps} rounds",
            "adjoint_ms": plain, "adjoint_params_ms": params, "adjoint_exact_ms": ex_ms,
            "exact_krylov_iterations": {"mean": float(its.mean()), "median": float(np.median(its)),
                                        "max": int(its.max()), "not_converged": int(((k >> 16) & 1).sum())},
            "outputs": f"dL/dk_p ({ctx.n_servo} servo gains), dL/dm ({ctx.nb} body masses), "
                       f"dL/dI ({3 * ctx.nb} principal moments), dL/dmu per world"}


def run_linear_solvers(args, torch, reps=3):
    """The Schur solve of Eq. (12) by the direct block-arrowhead factor against the paper's
    matrix-free PCR (Sec. III-C; 16 PCR iterations per Newton step in Sec. IV-B) with the
    Jacobi and the block-Jacobi preconditioner, on the robot over the box (args.worlds
    worlds) and the mesh terrain (args.terrain_worlds worlds, truncated pull-back), FP32,
    budget 16: per configuration the 10-step chunk (forward with the tape, then the
    adjoint, whose PCR solve runs to 1e-10), 2 warm-up and `reps` timed chunks; the share
    of steps whose Newton iteration met the tolerance within the budget, and the adjoint's
    PCR iterations."""
    from paper_2609_08800_gb300.ostrich import Context
    configs = [("direct", {}),
               ("pcr_jacobi_16", dict(linear_solver=S.LIN_PCR, precond=S.PC_JACOBI, pcr_iters=16)),
               ("pcr_block_16", dict(linear_solver=S.LIN_PCR, precond=S.PC_BLOCK, pcr_iters=16)),
               ("pcr_jacobi_64", dict(linear_solver=S.LIN_PCR, precond=S.PC_JACOBI, pcr_iters=64)),
               ("pcr_block_32", dict(linear_solver=S.LIN_PCR, precond=S.PC_BLOCK, pcr_iters=32))]
    out = {}
    legs = [("robot_over_box", args.worlds)]
    if args.terrain_worlds > 0:
        legs.append(("mesh_terrain", args.terrain_worlds))
    for leg, W in legs:
        if leg == "robot_over_box":
            scene, states, controls, g = make_inputs(W, seed=0)
            pull = S.PULLBACK_FULL
        else:
            scene = S.terrain_scene()
            states = S.terrain_states(scene, W, seed=0)
            knots = S.spline_knots(W, n_wheels=4, n_knots=8, seed=1)
            controls = np.ascontiguousarray(np.einsum("tk,wjk->tjw", SP.basis(100, 8, H), knots))[:CHUNK]
            controls = controls.astype(np.float32)
            g = np.zeros((scene.n_state, W))
            pull = S.PULLBACK_TRUNCATED
        res = {"worlds": W}
        for name, kw in configs:
            cfg = S.SolverConfig(tol=FP32_TOL, pullback=pull, **kw)
            ctx = Context(scene, cfg, W, dtype="f32", tape_slots=CHUNK, threads=64 if leg == "robot_over_box" else 128)
            kry = torch.zeros(W, dtype=torch.int32, device="cuda")
            ctx.set_adjoint_mode(0, kry)
            chunk = Chunk(ctx, torch, W)
            s0 = torch.tensor(states, dtype=torch.float32, device="cuda")
            ctl = torch.tensor(controls, dtype=torch.float32, device="cuda")
            gT = torch.tensor(g, dtype=torch.float32, device="cuda")
            if leg == "mesh_terrain":
                chunk.run(s0, ctl, gT)                      # landing, then chunks from the landed states
                s0 = chunk.states[CHUNK].clone()
                gT[0] = 2.0 * (s0[0] - 3.0)
                gT[1] = 2.0 * s0[1]
            for _ in range(2):
                chunk.run(s0, ctl, gT)
            torch.cuda.synchronize()
            evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(CHUNK)] for _ in range(reps)]
            eva = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(CHUNK)] for _ in range(reps)]
            for k in range(reps):
                chunk.run(s0, ctl, gT, evs[k], eva[k])
            torch.cuda.synchronize()
            it = np.stack([t.cpu().numpy() for t in chunk.iters]) & 0xFFFF
            step_ms = statistics.mean(e[0].elapsed_time(e[1]) for k in range(reps) for e in evs[k])
            adj_ms = statistics.mean(e[0].elapsed_time(e[1]) for k in range(reps) for e in eva[k])
            kr = kry.cpu().numpy()
            r = {"step_ms": step_ms, "adjoint_ms": adj_ms,
                 "world_steps_per_s": W * CHUNK / ((step_ms + adj_ms) * CHUNK * 1e-3),
                 "newton_iters_mean": float(it.mean()), "converged_within_budget": float((it < cfg.budget).mean())}
            if kw:
                r["adjoint_pcr_iters_mean"] = float((kr & 0xFFFF).mean())
                r["adjoint_pcr_not_converged"] = int(((kr >> 16) & 1).sum())
            res[name] = r
            ctx.close()
        out[leg] = res
    out["settings"] = "FP32, Newton budget 16, tol 1e-4 m/s, h = 0.1; robot 64 and terrain 128 threads per world, " \
                      "one CTA per world; adjoint PCR restarted on the true residual to |r| <= 1e-10 |b| (at most 256 iterations)"
    return out


def run_e2e(args, ctx, chunk, states, controls, g, torch):
    """Same chunk through the public API with pinned host buffers; copies inside the timing."""
    W = states.shape[1]
    hs = torch.tensor(states, dtype=torch.float32).pin_memory()
    hc = torch.tensor(controls, dtype=torch.float32).pin_memory()
    hg = torch.tensor(g, dtype=torch.float32).pin_memory()
    ds0 = torch.empty(ctx.n_state, W, dtype=torch.float32, device="cuda")
    dc = torch.empty_like(hc, device="cuda")
    dg = torch.empty_like(hg, device="cuda")
    out_state = torch.empty(ctx.n_state, W, dtype=torch.float32).pin_memory()
    out_grad = torch.empty(ctx.n_state, W, dtype=torch.float32).pin_memory()
    out_dctl = torch.empty(CHUNK, ctx.n_servo, W, dtype=torch.float32).pin_memory()

    def once():
        ds0.copy_(hs, non_blocking=True)
        dc.copy_(hc, non_blocking=True)
        dg.copy_(hg, non_blocking=True)
        chunk.run(ds0, dc, dg)
        out_state.copy_(chunk.states[CHUNK], non_blocking=True)
        out_grad.copy_(chunk.g[0], non_blocking=True)
        out_dctl.copy_(chunk.dctl, non_blocking=True)

    for _ in range(2):
        once()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = max(2, args.steps)
    a.record()
    for _ in range(n):
        once()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / n
    h2d = (hs.numel() + hc.numel() + hg.numel()) * 4
    d2h = (out_state.numel() + out_grad.numel() + out_dctl.numel()) * 4
    return {"value": W * CHUNK / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": ms}


def run_plain(args, scene, cfg, states, controls, g, torch):
    """One world per launch: W = 1 contexts over the same kernels, host loop over worlds."""
    from paper_2609_08800_gb300.ostrich import Context
    n = min(args.plain_worlds, states.shape[1])
    W = states.shape[1]
    ctx = Context(scene, cfg, 1, dtype="f32", tape_slots=CHUNK, ld=W)
    s0 = torch.tensor(states, dtype=torch.float32, device="cuda")
    ctl = torch.tensor(controls, dtype=torch.float32, device="cuda")
    gT = torch.tensor(g, dtype=torch.float32, device="cuda")
    st = [torch.empty_like(s0) for _ in range(CHUNK + 1)]
    gr = [torch.empty_like(s0) for _ in range(CHUNK + 1)]
    dctl = torch.empty_like(ctl)
    imp = torch.empty(ctx.m_max, W, dtype=torch.float32, device="cuda")
    st[0].copy_(s0)
    gr[CHUNK].copy_(gT)
    esz = 4

    class P:   # a device address with an element offset (column w of a dense [rows, ld] array)
        is_cuda = True

        def __init__(self, t, off):
            assert t.is_contiguous()
            self.p = t.data_ptr() + off * esz

        def data_ptr(self):
            return self.p

        def is_contiguous(self):
            return True

    def world(w):
        for t in range(CHUNK):
            ctx.ostrich_step(P(st[t], w), P(ctl[t], w), H, P(st[t + 1], w), P(imp, w), tape_slot=t)
        for t in reversed(range(CHUNK)):
            ctx.ostrich_adjoint(t, P(gr[t + 1], w), H, P(gr[t], w), P(dctl[t], w))

    for w in range(min(8, n)):
        world(w)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for w in range(n):
        world(w)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    ctx.close()
    return {"value": n * CHUNK / (ms * 1e-3), "unit": UNIT, "worlds_timed": n, "launches": 2 * CHUNK * n,
            "note": "same kernels, one world per launch (W = 1), host loop over worlds"}


def run_terrain(args, torch):
    """Mesh terrain (Sec. IV-D): 256 x 256 heightmap, FP32, truncated pull-back.  The
    robots are first rolled 10 steps from their drop so that they stand on the terrain;
    then 10-step chunks (forward with the tape, then the adjoint) are timed."""
    from paper_2609_08800_gb300 import tune
    from paper_2609_08800_gb300.ostrich import Context
    W = args.terrain_worlds
    scene = S.terrain_scene()
    states = S.terrain_states(scene, W, seed=0)
    knots = S.spline_knots(W, n_wheels=4, n_knots=8, seed=1)
    ctl_all = np.ascontiguousarray(np.einsum("tk,wjk->tjw", SP.basis(100, 8, H), knots)).astype(np.float32)
    cfg = S.SolverConfig(tol=FP32_TOL, pullback=S.PULLBACK_TRUNCATED)
    ctx = Context(scene, cfg, W, dtype="f32", tape_slots=CHUNK)
    threads = tune.apply(ctx) or 64
    schedule = getattr(ctx, "schedule", 0)
    chunk = Chunk(ctx, torch, W)
    s0 = torch.tensor(states, dtype=torch.float32, device="cuda")
    c0 = torch.tensor(ctl_all[:CHUNK], device="cuda")
    c1 = torch.tensor(ctl_all[CHUNK:2 * CHUNK], device="cuda")
    gT = torch.zeros(ctx.n_state, W, dtype=torch.float32, device="cuda")
    chunk.run(s0, c0, gT)                               # landing
    s1 = chunk.states[CHUNK].clone()
    gT[0] = 2.0 * (s1[0] - 3.0)
    gT[1] = 2.0 * s1[1]
    for _ in range(2):
        chunk.run(s1, c1, gT, record_ids=True)
    torch.cuda.synchronize()
    K = max(1, args.steps)
    evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(CHUNK)] for _ in range(K)]
    eva = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(CHUNK)] for _ in range(K)]
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for k in range(K):
        chunk.run(s1, c1, gT, evs[k], eva[k])
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / K
    iters = np.stack([t.cpu().numpy() for t in chunk.iters])
    ctx.close()
    return {"workload": f"mesh_terrain_{W}_worlds_fp32_fwd_adj_chunk10_truncated_pullback", "value": W * CHUNK / (ms * 1e-3),
            "unit": UNIT, "ms_per_chunk": ms, "threads_per_world": threads, "schedule": schedule,
            "step_ms_avg": statistics.mean(e[0].elapsed_time(e[1]) for k in range(K) for e in evs[k]),
            "adjoint_ms_avg": statistics.mean(e[0].elapsed_time(e[1]) for k in range(K) for e in eva[k]),
            "newton_iters_mean": float((iters & 0xFFFF).mean()), "active_rows_mean": float((iters >> 16).mean())}


def run_serving(args, torch):
    """The serving workload: a seeded Poisson stream (mean args.serve_rate req/s over args.serve_seconds of
    arrivals; 1-512 worlds log-uniform; horizon 20-200 steps; box-drop, robot-over-box and
    mesh-terrain scenes; half forward-only, half forward+adjoint) served by continuous
    batching, then the same stream by a FIFO queue of batched requests and by the plain
    form (one request at a time, one world per launch).  The stream offers more
    world-steps per second than the GPU serves, so every queue grows while arrivals last:
    each run stops at a wall-clock cutoff and reports its finished requests' p50/p99 and,
    counting the unfinished ones at their censored latency (cutoff - arrival), lower
    bounds on the stream's p50/p99.  Continuous batching is also run at
    args.serve_rate_stable req/s, a load within its capacity."""
    import time as _time
    from paper_2609_08800_gb300 import serve, tune
    cfg = S.SolverConfig(tol=FP32_TOL)
    pools = []
    kinds = ("box", "robot", "terrain")
    for kind in kinds:
        kcfg = S.SolverConfig(tol=FP32_TOL, pullback=S.PULLBACK_TRUNCATED) if kind == "terrain" else cfg
        p = serve.Pool(kind, kcfg, 8192, h=H, K=CHUNK, t_max=200, hbm_share=0.2)
        tune.apply(p.ctx)
        pools.append(p)
    warm = serve.poisson_stream(args.serve_rate, 0.05, seed=99, kinds=kinds, max_worlds=64, horizon=(20, 25))
    serve.Server(pools).run(warm)
    stated = serve.poisson_stream(args.serve_rate, args.serve_seconds, seed=0, kinds=kinds)
    offered = sum(r.n * r.T for r in stated) / args.serve_seconds
    out = {"stream": f"Poisson {args.serve_rate:g} req/s over {args.serve_seconds:g} s, seed 0, 1-512 worlds "
                     "(log-uniform), T 20-200, box-drop + robot-over-box + mesh terrain, half with adjoint",
           "requests_offered": len(stated), "offered_world_steps_per_s": offered}

    def timed(server, reqs, cutoff):
        for r in reqs:
            r.s0 = r.controls = None
        t0 = _time.perf_counter()
        done = server.run(reqs, t0=t0, deadline=cutoff)
        wall = _time.perf_counter() - t0
        st = serve.summarize(done, wall, getattr(server, "unfinished", ()), cutoff)
        st["wall_s"] = wall
        return st

    cb = serve.Server(pools)
    out["continuous_batching"] = timed(cb, stated, args.serve_seconds + args.serve_drain)
    out["continuous_batching"]["ticks"] = cb.tick
    stable = serve.poisson_stream(args.serve_rate_stable, args.serve_seconds_stable, seed=1, kinds=kinds)
    out["continuous_batching_within_capacity"] = dict(
        timed(serve.Server(pools), stable, args.serve_seconds_stable + args.serve_drain),
        stream=f"Poisson {args.serve_rate_stable:g} req/s over {args.serve_seconds_stable:g} s, seed 1, otherwise as above",
        offered_world_steps_per_s=sum(r.n * r.T for r in stable) / args.serve_seconds_stable)
    out["fifo_queue"] = timed(serve.Server(pools, fifo=True), serve.poisson_stream(args.serve_rate, args.serve_seconds,
                                                                                  seed=0, kinds=kinds),
                              args.serve_baseline_cutoff)
    out["plain_form"] = timed(serve.PlainServer(pools), serve.poisson_stream(args.serve_rate, args.serve_seconds,
                                                                            seed=0, kinds=kinds),
                              args.serve_baseline_cutoff)
    out["plain_form"]["note"] = "one request at a time, one world per launch (the same kernels with W = 1)"
    for p in pools:
        p.ctx.close()
    return out


def _oracle_opt_world(s0, knots, B, orc):
    """One world of the optimisation workload on the oracle: the T-step rollout under the
    spline controls B @ knots^T, the loss |p_xy(T) - (3, 0)|^2 of the chassis, then the
    backward sweep (every step re-solved by the oracle's adjoint call, as the checkpointed
    backward recomputes its segments) and the knot gradient B^T dL/dcontrols.  A world
    whose rollout diverged gets no gradient.  Returns (loss, dL/dknots [wheels, K])."""
    T = B.shape[0]
    ctl = B @ knots.T                                  # [T, wheels]
    traj = [np.asarray(s0, dtype=np.float64)]
    for t in range(T):
        traj.append(orc.step(traj[-1], ctl[t], H)["state"])
    sT = traj[T]
    loss = (sT[0] - 3.0) ** 2 + sT[1] ** 2
    if not np.isfinite(loss):
        return float(loss), np.zeros_like(knots)
    g = np.zeros_like(sT)
    g[0], g[1] = 2.0 * (sT[0] - 3.0), 2.0 * sT[1]
    du = np.zeros_like(ctl)
    for t in reversed(range(T)):
        r = orc.step_adjoint(traj[t], ctl[t], H, g)
        g, du[t] = r["dstate"], r["dubar"]
    return float(loss), np.nan_to_num((B.T @ du).T, nan=0.0, posinf=0.0, neginf=0.0)


_WORKER_ORACLE = None


def _worker_init():
    global _WORKER_ORACLE
    from oracle import oracle as O
    _WORKER_ORACLE = O.Oracle(S.robot_box_scene(), S.SolverConfig(tol=FP32_TOL))


def _worker_run(job):
    states, knots = job
    B = SP.basis(OPT_T, knots.shape[2], H)
    return [_oracle_opt_world(states[:, w], knots[w], B, _WORKER_ORACLE) for w in range(states.shape[1])]


class OracleOptSample:
    """The optimisation workload (robot over the box, 8-knot wheel splines, T = 100,
    h = 0.1, Newton budget 16, tol 1e-4, Adam with lr 0.3 on the knots) on a sample of
    worlds, on the FP64 oracle: in this process (procs = 1) or split over `procs` spawned
    processes, one oracle each (pool start-up and a one-world warm call outside the
    timing).  One call of `iteration` is one Adam iteration over the sample."""

    def __init__(self, n_worlds, procs=1):
        scene = S.robot_box_scene()
        self.n, self.procs = n_worlds, max(1, procs)
        self.states = S.robot_box_states(scene, n_worlds, seed=0).astype(np.float32).astype(np.float64)
        self.knots = S.spline_knots(n_worlds, n_wheels=4, n_knots=8, seed=0).astype(np.float32).astype(np.float64)
        self.m1, self.m2, self.t = np.zeros_like(self.knots), np.zeros_like(self.knots), 0
        self.pool, self.orc = None, None
        if self.procs > 1:
            import multiprocessing as mp
            self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_worker_init)
            self.pool.map(_worker_run, [(self.states[:, :1], self.knots[:1, :, :])] * self.procs)
        else:
            from oracle import oracle as O
            self.orc = O.Oracle(scene, S.SolverConfig(tol=FP32_TOL))
            B = SP.basis(OPT_T, self.knots.shape[2], H)
            self.orc.step(self.states[:, 0], B[0] @ self.knots[0].T, H)

    def iteration(self):
        """One Adam iteration over the sample; returns (world-steps, seconds)."""
        t0 = time.perf_counter()
        if self.pool is not None:
            bounds = np.linspace(0, self.n, self.procs + 1).astype(int)
            jobs = [(self.states[:, a:b], self.knots[a:b]) for a, b in zip(bounds[:-1], bounds[1:])]
            res = [r for part in self.pool.map(_worker_run, jobs) for r in part]
        else:
            B = SP.basis(OPT_T, self.knots.shape[2], H)
            res = [_oracle_opt_world(self.states[:, w], self.knots[w], B, self.orc) for w in range(self.n)]
        grad = np.stack([r[1] for r in res])
        # Adam (lr 0.3, betas 0.9 / 0.999, eps 1e-8), as torch.optim.Adam
        self.t += 1
        self.m1 = 0.9 * self.m1 + 0.1 * grad
        self.m2 = 0.999 * self.m2 + 0.001 * grad * grad
        mh, vh = self.m1 / (1.0 - 0.9 ** self.t), self.m2 / (1.0 - 0.999 ** self.t)
        self.knots = self.knots - 0.3 * mh / (np.sqrt(vh) + 1e-8)
        return self.n * OPT_T, time.perf_counter() - t0

    def describe(self, dt):
        how = f"{self.procs} processes, one oracle each" if self.pool is not None else "single thread"
        return (f"{self.n} worlds x one Adam iteration over T = {OPT_T} (forward rollout, then every step "
                f"re-solved with its adjoint, then the knot update), {how}, {dt:.1f} s")

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()


def run_cpu_baseline(args):
    """FP64 oracle on one host thread: one Adam iteration of the optimisation workload on a
    bounded sample of args.cpu_worlds worlds."""
    smp = OracleOptSample(max(1, args.cpu_worlds), procs=1)
    n, dt = smp.iteration()
    return {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": smp.describe(dt)}


def opt_config(W):
    """The optimisation workload's `config` (both arms)."""
    return {"workload": f"robot_over_box_{W}_worlds_fp32_adam_T{OPT_T}_ckpt{CHUNK}",
            "worlds_per_gpu": W, "horizon_steps": OPT_T, "h": H, "checkpoint_every": CHUNK,
            "step": "one Adam iteration (lr 0.3) on 8-knot wheel splines: T forward steps, the backward's "
                    "recomputed steps and T adjoint steps; world-steps = W x T per iteration",
            "newton_budget": S.SolverConfig().budget, "tol": FP32_TOL}


# ---------------------------------------------------------------------------
# distributed helpers (replicas; the only collectives are the timing barrier/max)
# ---------------------------------------------------------------------------
_DIST = None


def dist_init():
    global _DIST
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("OSTRICH_BENCH_GLOO") is None else "gloo")
        _DIST = dist
    return int(os.environ.get("RANK", "0")), ws, int(os.environ.get("LOCAL_RANK", "0"))


def dist_barrier():
    if _DIST is not None:
        _DIST.barrier()


def dist_max(x):
    if _DIST is None:
        return x
    import torch
    dev = "cuda" if _DIST.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    _DIST.all_reduce(t, op=_DIST.ReduceOp.MAX)
    return float(t.item())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20, help="timed optimisation iterations (Adam iterations on the spline knots)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--worlds", type=int, default=8192)
    ap.add_argument("--terrain-worlds", type=int, default=2048, help="worlds of the mesh-terrain leg (0: skip)")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="arrival window of the serving stream (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-drain", type=float, default=30.0,
                    help="seconds allowed after the arrival window before a continuous-batching run is cut off")
    ap.add_argument("--serve-rate-stable", type=float, default=50.0, help="a request rate within capacity")
    ap.add_argument("--serve-seconds-stable", type=float, default=30.0)
    ap.add_argument("--serve-baseline-cutoff", type=float, default=20.0,
                    help="wall-clock cutoff of the FIFO-queue and plain-form runs of the stated stream")
    ap.add_argument("--threads", type=int, default=None, help="threads per world (default: autotuner table)")
    ap.add_argument("--linear-solvers", type=int, default=1,
                    help="1: time the direct factor against PCR (robot and terrain legs); 0: skip")
    ap.add_argument("--plain-worlds", type=int, default=512)
    ap.add_argument("--cpu-worlds", type=int, default=48,
                    help="worlds of the cpu_baseline sample (one Adam iteration on one host thread)")
    ap.add_argument("--ref-worlds", type=int, default=8,
                    help="worlds per process of the reference arm's sample (each step one Adam iteration)")
    ap.add_argument("--cpu-procs", type=int, default=0,
                    help="processes for the reference arm's oracle (0: all host cores)")
    ap.add_argument("--skip-extras", action="store_true",
                    help="time the batched kernels only (no e2e, plain-form or CPU legs); profiling runs")
    args = ap.parse_args()
    rank, ws, local_rank = dist_init()
    if args.impl == "reference":
        if rank != 0:
            return
        procs = max(1, args.cpu_procs or (os.cpu_count() or 1))
        smp = OracleOptSample(args.ref_worlds * procs, procs=procs)
        for _ in range(args.warmup):
            smp.iteration()
        runs = [smp.iteration() for _ in range(args.steps)]
        smp.close()
        vals = [n / dt for n, dt in runs]
        v = statistics.median(vals)
        dt_med = statistics.median(dt for _, dt in runs)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * dt_med,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": dict(opt_config(args.worlds), sample_worlds=smp.n,
                               parallelism=f"oracle on {procs} host processes"),
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle",
                                 "sample": smp.describe(dt_med) + " (median step)"},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    out = run_ours(args, rank, ws, local_rank)
    if rank == 0:
        print(json.dumps(out))
    if _DIST is not None:
        _DIST.destroy_process_group()


if __name__ == "__main__":
    main()
