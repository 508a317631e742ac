"""Autotuner for the launch shape: threads per world (32, 64 or 128) and the schedule
(one CTA per world, or persistent CTAs taking the heaviest worlds first).

One CTA steps one world; its threads split the rows of the Schur blocks, the
row-parallel solves and the per-body reductions.  More threads shorten each phase
but cut the CTAs resident per SM (registers) and add barrier cost, so the best
count depends on the row count m (hence the workspace) and the precision.  The
tuner times one step launch per candidate on the caller's own states and keeps the
fastest in a table keyed by (precision, m-bucket, device), persisted as JSON:
first the user's table (OSTRICH_AUTOTUNE_CACHE, default ~/.cache/ostrich), then the
table shipped beside this module.
"""
from __future__ import annotations

import json
import os
from pathlib import Path

import torch

CANDIDATES = (32, 64, 128)
SHIPPED = Path(__file__).with_name("autotune.json")


def cache_path():
    return Path(os.environ.get("OSTRICH_AUTOTUNE_CACHE", Path.home() / ".cache" / "ostrich" / "autotune.json"))


def m_bucket(m_max):
    """Row-count bucket: multiples of 32 rows (box 12 -> 32, robot 120 -> 128, 216 -> 224)."""
    return 32 * ((int(m_max) + 31) // 32)


def key(ctx, device=None):
    prec = "f64" if ctx.dtype == torch.float64 else "f32"
    name = torch.cuda.get_device_name(device).replace(" ", "_")
    return f"{prec}:m{m_bucket(ctx.m_max)}:{name}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def lookup_entry(ctx):
    k = key(ctx)
    for path in (cache_path(), SHIPPED):
        entry = _load(path).get(k)
        if entry:
            return entry
    return None


def lookup(ctx):
    entry = lookup_entry(ctx)
    return int(entry["threads"]) if entry else None


def store(k, entry, path=None):
    path = Path(path or cache_path())
    path.parent.mkdir(parents=True, exist_ok=True)
    table = _load(path)
    table[k] = entry
    tmp = path.with_suffix(".tmp")
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_step(ctx, state, controls, h, reps=3, stream=None):
    """Mean device time (ms) of one step launch over `reps` launches after one warm-up."""
    stream = stream or torch.cuda.current_stream()
    out = torch.empty_like(state)
    with torch.cuda.stream(stream):
        ctx.ostrich_step(state, controls, h, out, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ctx.ostrich_step(state, controls, h, out, stream=stream)
        e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


SCHEDULES = (0, 1)


def tune(ctx, state, controls, h, candidates=CANDIDATES, reps=3, persist=True, path=None, schedules=SCHEDULES):
    """Time each (threads, schedule) candidate on (state, controls), set the fastest on ctx,
    record it.  Returns (best threads, {threads: ms} at the best schedule)."""
    times = {}
    for sch in schedules:
        ctx.set_schedule(sch)
        for t in candidates:
            ctx.set_threads(t)
            times[(t, sch)] = time_step(ctx, state, controls, h, reps)
    best_t, best_s = min(times, key=times.get)
    ctx.set_threads(best_t)
    ctx.set_schedule(best_s)
    if persist:
        store(key(ctx), {"threads": best_t, "schedule": best_s,
                         "ms": {f"{t}/{sch}": round(v, 4) for (t, sch), v in times.items()},
                         "worlds": ctx.n_worlds}, path)
    return best_t, {t: v for (t, sch), v in times.items() if sch == best_s}


def apply(ctx):
    """Set the tabled thread count and schedule on ctx if the table has them; returns the
    thread count (or None)."""
    entry = lookup_entry(ctx)
    if entry is None:
        return None
    ctx.set_threads(int(entry["threads"]))
    ctx.set_schedule(int(entry.get("schedule", 0)))
    return int(entry["threads"])


def main(argv=None):
    """Tune the box-drop and robot-over-box scenes in both precisions and write the table
    (python -m paper_2609_08800_gb300.tune --out FILE)."""
    import argparse

    import numpy as np

    from . import scenes as S
    from .ostrich import Context

    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=str(cache_path()))
    ap.add_argument("--worlds", type=int, default=8192)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args(argv)
    W, h = args.worlds, 0.1
    cases = []
    box = S.box_drop_scene()
    cases.append((box, np.repeat(S.box_drop_state(box, 0.3), W, axis=1), np.zeros((1, W))))
    rob = S.robot_box_scene()
    cases.append((rob, S.robot_box_states(rob, W, seed=0), S.random_controls(rob.n_servos, W, seed=0, low=-3, high=3)))
    ter = S.terrain_scene()
    Wt = min(W, 2048)
    st = S.terrain_states(ter, Wt, seed=0)
    st[2:7 * ter.n_bodies:7] -= 0.012                    # resting on the terrain
    cases.append((ter, st, S.random_controls(ter.n_servos, Wt, seed=0, low=-3, high=3)))
    for scene, st, ub in cases:
        for prec in ("f32", "f64"):
            dt = torch.float64 if prec == "f64" else torch.float32
            try:
                ctx = Context(scene, S.SolverConfig(tol=1e-4 if prec == "f32" else 1e-5), st.shape[1], dtype=prec)
            except RuntimeError as e:                    # e.g. FP64 terrain exceeds shared memory
                print(scene.name, prec, "skipped:", e)
                continue
            best, times = tune(ctx, torch.tensor(st, dtype=dt, device="cuda"), torch.tensor(ub, dtype=dt, device="cuda"),
                               h, reps=args.reps, path=args.out)
            print(key(ctx), best, ctx.schedule, {t: round(v, 3) for t, v in times.items()})
            ctx.close()


if __name__ == "__main__":
    main()
