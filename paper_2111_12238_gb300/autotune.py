"""Autotuner of the executor's launch shape.

For one schedule and one way of running it, times candidate (lanes per row, items per
partition) pairs on the GPU and keeps the fastest. A candidate is applied without
re-inspecting: ``sf_schedule_recut`` re-cuts the partitions for the new cost target
(items per partition x mean vertex cost) and lane count, keeping levels and order.
Results are cached in a JSON file (``SF_TUNE_CACHE``, default
``~/.cache/sparsefusion/tune.json``) keyed by the schedule's shape and the GPU's name.
"""
from __future__ import annotations

import json
import os
import time
from typing import Callable, Dict, Iterable, Optional, Sequence, Tuple

import torch

from . import sparsefusion as sf

DEFAULT_LANES = (1, 2, 4, 8, 16, 32)
DEFAULT_ITEMS = (2, 4, 8, 16, 32)
DEFAULT_TEAMS = (8, 32)


def _cache_path() -> str:
    return os.environ.get("SF_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "sparsefusion",
                                                        "tune.json"))


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(path, data):
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def signature(sched: sf.Schedule, which: int, dtype: torch.dtype, k: int) -> str:
    inf = sched.info()
    nv = inf["n_items"] if which == 0 else inf["adj_n_items"]
    cost = inf["cost_total"] if which == 0 else inf["adj_cost_total"]
    depth = inf["depth"] if which == 0 else inf["adj_depth"]
    dev = torch.cuda.get_device_name()
    return (f"{sched.pair}|dir={which}|n={inf['n']}|items={nv}|cost={cost}|depth={depth}|inst={inf['instances']}"
            f"|k={k}|{str(dtype).replace('torch.', '')}|{dev}")


def _time(run: Callable[[], object], reps: int) -> float:
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    run()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        start.record()
        run()
        end.record()
        end.synchronize()
        times.append(start.elapsed_time(end))
    times.sort()
    return times[len(times) // 2]


def tune(sched: sf.Schedule, run: Callable[[], object], *, which: int = 0, dtype: torch.dtype = torch.float64,
         k: int = 1, lanes: Sequence[int] = DEFAULT_LANES, items: Sequence[int] = DEFAULT_ITEMS,
         teams: Sequence[int] = DEFAULT_TEAMS, reps: int = 3,
         budget_s: float = 20.0, use_cache: bool = True) -> Dict:
    """Chooses lanes per row, team width and items per partition for `which` (0 forward, 1 adjoint) of
    `sched`, timing `run()` (one execution) for every candidate within `budget_s` seconds.
    Leaves the schedule cut and launched with the best candidate and returns
    dict(lanes, items, team, part_cost_target, ms, trials, cached)."""
    inf = sched.info()
    nv = inf["n_items"] if which == 0 else inf["adj_n_items"]
    cost_total = inf["cost_total"] if which == 0 else inf["adj_cost_total"]
    mean = max(1, -(-cost_total // max(nv, 1)))
    kt = 1
    while kt < k and kt < 32:
        kt *= 2
    path = _cache_path()
    key = signature(sched, which, dtype, k)
    cache = _load_cache(path) if use_cache else {}
    if use_cache and key in cache:
        best = cache[key]
        sched.recut(which, best["part_cost_target"], best["lanes"], best.get("team", 0))
        return dict(best, cached=True)
    cands = [(L, p, T) for L in lanes if L >= kt for T in teams if T >= L for p in items
             if p <= max(1, T // L) * 4]
    # start from the default shape, then the rest
    cands.sort(key=lambda c: (abs(c[0] - max(1, kt)), c[2] != 32, abs(c[1] - 8)))
    t0 = time.perf_counter()
    trials = []
    best = None
    for L, p, T in cands:
        if trials and time.perf_counter() - t0 > budget_s:
            break
        C = max(1, p * mean)
        sched.recut(which, C, L, T)
        ms = _time(run, reps)
        sched.check()
        trials.append({"lanes": L, "items": p, "team": T, "part_cost_target": C, "ms": ms})
        if best is None or ms < best["ms"]:
            best = trials[-1]
    sched.recut(which, best["part_cost_target"], best["lanes"], best["team"])
    if use_cache:
        cache = _load_cache(path)
        cache[key] = best
        _store_cache(path, cache)
    return dict(best, cached=False, trials=trials)
