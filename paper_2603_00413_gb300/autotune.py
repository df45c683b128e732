"""Autotuner of the library's launch and scheduling knobs.

The kernels' results do not depend on the knobs (the same closest hits are
found), only their speed does: node format of the traversal (binary or
4-wide), the width of the traversal-order buckets (0: append order),
resident traversal CTAs per SM (its register budget), node visits
per scheduling round and the idle-lane count that triggers a refill, and the
grid of the shading and adjoint kernels.  `tune` times a caller's step
function under a grid of settings with CUDA events and keeps the fastest;
results are cached per device and workload key in a JSON file, so a workload
is tuned once per machine.
"""
from __future__ import annotations

import itertools
import json
import os

import torch

from . import get_tuning, set_tuning

DEFAULT_SPACE = {
    "bvh_width": (2, 4),
    "trace_order": (0, 16, 20, 22),
    "trace_blocks_per_sm": (4, 5, 6),
    "trace_steps": (32, 64, 128, 192, 256),
    "trace_refill": (4, 8, 16),
    "shade_blocks_per_sm": (4, 8, 16),
}

CACHE_PATH = os.path.join(os.path.expanduser("~"), ".cache", "difftrans_gb300_tuning.json")


def _time(step, reps: int) -> float:
    step()  # warm (first launches, caches)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        step()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def tune(step, key: str, space: dict = None, reps: int = 2, cache_path: str = CACHE_PATH, retune: bool = False,
         coordinate: bool = True) -> dict:
    """Find the fastest knob setting for `step` (a callable running one
    piece of work on the current stream) and leave it set.

    coordinate=True tunes one knob at a time in the order of `space`
    (starting from the current settings), which takes the sum rather than
    the product of the option counts; False sweeps the full product.
    Returns {"tuning": {...}, "ms": best time, "trials": [...]}."""
    dev = torch.cuda.get_device_name()
    full_key = f"{dev}|{key}"
    cache = _load_cache(cache_path)
    if not retune and full_key in cache:
        set_tuning(**cache[full_key]["tuning"])
        return cache[full_key]
    space = dict(DEFAULT_SPACE if space is None else space)
    best = get_tuning()
    trials = []
    best_ms = _time(step, reps)
    trials.append((dict(best), best_ms))
    if coordinate:
        for knob, options in space.items():
            start = best[knob]  # the incumbent, already timed
            for v in options:
                if v == start:
                    continue
                cand = dict(best)
                cand[knob] = v
                set_tuning(**cand)
                ms = _time(step, reps)
                trials.append((dict(cand), ms))
                if ms < best_ms:
                    best, best_ms = cand, ms
            set_tuning(**best)
    else:
        names = list(space)
        for combo in itertools.product(*[space[n] for n in names]):
            cand = dict(best)
            cand.update(dict(zip(names, combo)))
            set_tuning(**cand)
            ms = _time(step, reps)
            trials.append((dict(cand), ms))
            if ms < best_ms:
                best, best_ms = dict(cand), ms
    set_tuning(**best)
    result = {"tuning": best, "ms": best_ms, "trials": [{"tuning": t, "ms": m} for t, m in trials]}
    try:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        cache = _load_cache(cache_path)
        cache[full_key] = result
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return result
