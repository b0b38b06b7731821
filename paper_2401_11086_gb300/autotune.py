"""Persisted launch schedules for libsmrt's 1D-line kernels.

lb_autotune (C++) times the candidate schedules of a context and applies the fastest. This
module stores the result in a JSON file keyed by the GPU, velocity set, order, precision and
the instance lengths, so that later runs of the same workload apply it without re-timing.
The file is $SMRT_SCHEDULE_CACHE, else ~/.cache/smrt/schedules.json.
"""
from __future__ import annotations

import hashlib
import json
import os

from . import api


def cache_path() -> str:
    return os.environ.get("SMRT_SCHEDULE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "smrt", "schedules.json"))


def schedule_key(ctx: api.Context, lengths) -> str:
    import torch
    gpu = torch.cuda.get_device_name(ctx.device)
    h = hashlib.sha256(",".join(str(int(L)) for L in lengths).encode()).hexdigest()[:16]
    return f"{gpu}|q{ctx.lattice.q}|N{ctx.N}|p{ctx.precision}|{len(lengths)}x{h}"


def _load(path: str) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _tune_persistent(ctx: api.Context, fa, fb, trial_steps: int) -> dict:
    """Time every persistent schedule (tile widths 32/64/128; 1, 2, 4 or all resident blocks
    per SM) by an lb_step of trial_steps steps (one cooperative launch, as a graph replays it)
    and apply the fastest."""
    import torch
    stream = ctx.stream if ctx.stream is not None else torch.cuda.current_stream(ctx.device)
    best = None
    for width in (32, 64, 128):
        for bps in (0, 1, 2, 4):
            try:
                api.lb_set_schedule(ctx, width, bps, 1)
            except api.SmrtError:
                continue
            api.lb_step(ctx, fa, fb, 2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            n = trial_steps + (trial_steps & 1)
            e0.record(stream)
            api.lb_step(ctx, fa, fb, n)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / n
            if best is None or ms < best["ms_per_step"]:
                best = {"tile_width": width, "blocks_per_sm": bps, "persistent": 1, "tensor_cores": 0,
                        "ms_per_step": ms}
    if best is None:
        raise RuntimeError("no persistent schedule can be resident on this context")
    api.lb_set_schedule(ctx, best["tile_width"], best["blocks_per_sm"], 1)
    return best


def tuned_schedule(ctx: api.Context, f, lengths, trial_steps: int = 20, path: str | None = None,
                   retune: bool = False, persistent: bool = False) -> dict:
    """Apply the cached schedule for this workload, or autotune on copies of the state f (f is
    left untouched) and cache the winner. persistent: choose among the persistent schedules
    only (what lb_step_graph replays). Returns the schedule applied."""
    path = path or cache_path()
    key = schedule_key(ctx, lengths) + ("|persistent" if persistent else "")
    db = _load(path)
    if key in db and not retune:
        s = db[key]
        api.lb_set_schedule(ctx, s["tile_width"], s["blocks_per_sm"], s["persistent"], s.get("tensor_cores", 0))
        return s
    fa, fb = f.clone(), ctx.new_state()
    best = _tune_persistent(ctx, fa, fb, trial_steps) if persistent else api.lb_autotune(ctx, fa, fb, trial_steps)
    db[key] = best
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(db, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return best
