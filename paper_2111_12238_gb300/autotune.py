"""Autotuner of the executor's launch shape.

For one schedule and one way of running it, times candidate launch shapes on the GPU and
keeps the fastest: for one right-hand side the row-block executors (warp-specialised with
cp.async or with packed records and bulk copies, and the plain one) with several block sizes
(and lane counts), and the partition executor with several (lanes per row, team width, items
per partition), then, for separated schedules, the best shape with the second kernel's
vertices placed later (``sf_schedule_replace``), the best partition shape on the executor's
occupancy variants (``sf_schedule_set_occupancy``) and with the teams split between the two
partition classes (``sf_schedule_set_split``), for several right-hand sides with other
right-hand-side tiles (``sf_schedule_set_rhs_tile``), and with long rows split over several
teams at several costs per slice (``sf_schedule_set_slices``). Candidates are applied without
re-inspecting: ``sf_schedule_reblock``
rebuilds the row-block order, ``sf_schedule_recut`` re-cuts the partitions for a new cost
target (items per partition x mean vertex cost); levels are kept.
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
DEFAULT_ITEMS = (1, 2, 4, 8, 16, 32)
DEFAULT_TEAMS = (8, 32)
DEFAULT_BLOCK_ROWS = (1024, 2048, 4096, 8192, 16384)
DEFAULT_BLOCK_LANES = (1, 2, 4, 32)
DEFAULT_SPLITS = (50, 65, 80, 90)
DEFAULT_PLACEMENTS = (-1, 2, 8, 32)
DEFAULT_RHS_TILES = (1, 2, 4, 8, 16, 32)
DEFAULT_SLICES = (32, 64, 128, 256, 512)


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


def _apply(sched: sf.Schedule, which: int, c: Dict, mean: int):
    """Applies one candidate launch shape to direction `which` of the schedule."""
    sched.replace(which, c.get("g2", 0))   # no-op unless the placement changes
    sched.set_occupancy(which, c.get("occ", 1))
    sched.set_rhs_tile(which, c.get("rt", 0))
    sched.set_slices(which, c.get("slices", 0) if c["exec"] == "partitions" else 0)
    if sched.pair == "spmv_trsv" and which == 0:
        sched.set_packing(c.get("packing", 1))
    if c["exec"] == "cta":
        sched.reblock(which, 0, 5, c.get("cps", 0))
        sched.set_split(which, 0)
    elif c["exec"] == "blocks":
        sched.reblock(which, c["block_rows"], 2, c["block_lanes"])
        sched.set_split(which, 0)
    elif c["exec"] in ("ws", "tma"):
        sched.reblock(which, c["block_rows"], 3 if c["exec"] == "ws" else 4, 0)
        sched.set_split(which, 0)
    else:
        c["part_cost_target"] = max(1, c["items"] * mean)
        sched.recut(which, c["part_cost_target"], c["lanes"], c["team"])
        sched.reblock(which, 0, 1, 0)
        sched.set_split(which, c.get("split", 0))


def tune(sched: sf.Schedule, run: Callable[[], object], *, which: int = 0, dtype: torch.dtype = torch.float64,
         k: int = 1, lanes: Sequence[int] = DEFAULT_LANES, items: Sequence[int] = DEFAULT_ITEMS,
         teams: Sequence[int] = DEFAULT_TEAMS, blocks: bool = True,
         block_rows: Sequence[int] = DEFAULT_BLOCK_ROWS, block_lanes: Sequence[int] = DEFAULT_BLOCK_LANES,
         splits: Sequence[int] = DEFAULT_SPLITS, placements: Sequence[int] = DEFAULT_PLACEMENTS, occupancy=True,
         rhs_tiles: Sequence[int] = DEFAULT_RHS_TILES, slices: Sequence[int] = DEFAULT_SLICES,
         packing: bool = True, reps: int = 3, budget_s: float = 20.0,
         use_cache: bool = True) -> Dict:
    """Chooses the executor and its launch shape for `which` (0 forward, 1 adjoint) of
    `sched`, timing `run()` (one execution) for every candidate within `budget_s` seconds.
    Leaves the schedule set to the best candidate and returns it as a dict (exec, its
    parameters, ms) with the list of trials and whether it came from the cache."""
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
        _apply(sched, which, best, mean)
        return dict(best, cached=True)
    # partition shapes first (the default executor; they finish the budget with a sound
    # choice), then the row-block executors
    pc = [(L, p, T) for L in lanes if L >= kt for T in teams if T >= L for p in items if p <= max(1, T // L) * 4]
    pc.sort(key=lambda c: (abs(c[0] - max(1, kt)), c[2] != 32, abs(c[1] - 8)))
    cands = [{"exec": "partitions", "lanes": L, "items": p, "team": T} for L, p, T in pc]
    if k == 1 and blocks and sched.pair in ("trsv_spmv", "trsv") and which == 0 and \
            (inf["instances"] > 1 or inf["n"] <= 65536):
        # small systems, or batches of independent instances: one CTA per instance, x on chip
        cps = (2, 1, 4) if inf["instances"] > 1 else (1,)
        cands[1:1] = [{"exec": "cta", "cps": c} for c in cps]
    if k == 1 and blocks:
        n = inf["n"]
        sizes = [B for B in block_rows if B <= 2 * max(n, 1)]
        cands += [{"exec": "ws", "block_rows": B} for B in sizes]
        cands += [{"exec": "tma", "block_rows": B} for B in sizes]
        cands += [{"exec": "blocks", "block_rows": B, "block_lanes": L} for B in sizes for L in block_lanes]
    t0 = time.perf_counter()
    trials = []
    best = None
    for c in cands:
        if trials and time.perf_counter() - t0 > budget_s:
            break
        try:
            _apply(sched, which, c, mean)
            ms = _time(run, reps)
        except sf.SparseFusionError:
            # a row-block size whose shared-memory footprint does not fit this direction
            if c["exec"] not in ("blocks", "ws", "tma", "cta"):
                raise
            continue
        sched.check()
        trials.append(dict(c, ms=ms))
        if best is None or ms < best["ms"]:
            best = trials[-1]
    separated = inf["parts_class0" if which == 0 else "adj_parts_class0"] > 0
    # separated schedules: the best shape, and the best row-block shape, with the second
    # kernel's vertices placed later (slack, section 3.2.2); then the best partition shape
    # with the teams split between the two partition classes
    if best is not None and separated and placements:
        bases = [best]
        rb = [t for t in trials if t["exec"] in ("ws", "tma", "blocks", "cta")]
        if rb:
            rb_best = min(rb, key=lambda t: t["ms"])
            if rb_best is not best:
                bases.append(rb_best)
        shapes = [(b, g2) for b in bases for g2 in placements]
        for base, g2 in shapes:
            c = {kk: v for kk, v in base.items() if kk not in ("ms", "part_cost_target", "cached")}
            c["g2"] = g2
            try:
                _apply(sched, which, c, mean)
                ms = _time(run, reps)
            except sf.SparseFusionError:
                if c["exec"] not in ("blocks", "ws", "tma", "cta"):
                    raise
                continue
            sched.check()
            trials.append(dict(c, ms=ms))
            if ms < best["ms"]:
                best = trials[-1]
    # the best partition shape on the occupancy variants of the executor kernels
    ic0 = sched.pair in ("ic0", "ic0_trsv")
    occ_variant = (k == 1 and best is not None and best.get("lanes", 32) <= 4) or \
        (ic0 and best is not None and best.get("lanes") == 32 and best.get("team") == 32)
    if best is not None and best["exec"] == "partitions" and occupancy and occ_variant:
        c = {kk: v for kk, v in best.items() if kk in ("exec", "lanes", "items", "team", "g2")}
        c["occ"] = 3
        _apply(sched, which, c, mean)
        ms = _time(run, reps)
        sched.check()
        trials.append(dict(c, ms=ms))
        if ms < best["ms"]:
            best = trials[-1]
    # wide rows with value flags (16 or 32 lanes): the two-block variants, twice the teams
    if best is not None and best["exec"] == "partitions" and occupancy and not ic0 and \
            best.get("lanes", 0) >= 16:
        c = {kk: v for kk, v in best.items() if kk in ("exec", "lanes", "items", "team", "g2", "rt")}
        c["occ"] = 2
        _apply(sched, which, c, mean)
        ms = _time(run, reps)
        sched.check()
        trials.append(dict(c, ms=ms))
        if ms < best["ms"]:
            best = trials[-1]
    # several right-hand sides: the best partition shape with the other right-hand-side tiles
    # (lanes at least the tile; 16 or more lanes publish rows through their values)
    if best is not None and best["exec"] == "partitions" and k > 1 and rhs_tiles:
        base = {kk: v for kk, v in best.items() if kk in ("exec", "lanes", "items", "team", "g2", "occ")}
        for rt in rhs_tiles:
            if rt == kt or rt > 32:
                continue
            for L in sorted({max(base["lanes"], rt), 32}):
                c = dict(base, rt=rt, lanes=L, team=max(base["team"], L))
                if c["items"] > max(1, c["team"] // L) * 4:
                    c["items"] = max(1, c["team"] // L)
                _apply(sched, which, c, mean)
                ms = _time(run, reps)
                sched.check()
                trials.append(dict(c, ms=ms))
                if ms < best["ms"]:
                    best = trials[-1]
    # long rows split over several teams at several costs per slice
    if best is not None and best["exec"] == "partitions" and slices:
        base = {kk: v for kk, v in best.items() if kk in ("exec", "lanes", "items", "team", "g2", "occ", "rt")}
        bases = [base]
        if k > 1 and base.get("rt", kt) != kt:
            # one pass over the columns (the widest tile) at the same lanes
            bases.append({kk: v for kk, v in base.items() if kk != "rt"})
        if k > 1 and base.get("lanes") != 32:
            bases.append(dict({kk: v for kk, v in base.items() if kk != "rt"}, lanes=32, team=32, items=1))
        for b_, sc in [(b_, sc) for b_ in bases for sc in slices]:
            c = dict(b_, slices=sc)
            _apply(sched, which, c, mean)
            inf2 = sched.info()
            if (inf2["slice_units"] if which == 0 else inf2["adj_slice_units"]) == 0:
                continue   # nothing to split at this cost (or a kind that is not split)
            ms = _time(run, reps)
            sched.check()
            trials.append(dict(c, ms=ms))
            if ms < best["ms"]:
                best = trials[-1]
    # SpMV -> SpTRSV: separated packing (r = b - A x_in first, §3.2.3) on the best partition shape
    if best is not None and best["exec"] == "partitions" and sched.pair == "spmv_trsv" and which == 0 and packing:
        c = {kk: v for kk, v in best.items()
             if kk in ("exec", "lanes", "items", "team", "g2", "occ", "rt", "slices")}
        c["packing"] = 0
        if c.get("occ") == 3:
            c.pop("occ")   # the three-block kernels do not run separated packing
        try:
            _apply(sched, which, c, mean)
            ms = _time(run, reps)
            sched.check()
            trials.append(dict(c, ms=ms))
            if ms < best["ms"]:
                best = trials[-1]
        except sf.SparseFusionError:
            pass   # a launch that does not publish through values
    if best is not None and best["exec"] == "partitions" and splits and separated:
        for pct in splits:
            c = {kk: v for kk, v in best.items()
                 if kk in ("exec", "lanes", "items", "team", "g2", "occ", "rt", "slices")}
            c["split"] = pct
            _apply(sched, which, c, mean)
            ms = _time(run, reps)
            sched.check()
            trials.append(dict(c, ms=ms))
            if ms < best["ms"]:
                best = trials[-1]
    _apply(sched, which, best, mean)
    if use_cache:
        cache = _load_cache(path)
        cache[key] = best
        _store_cache(path, cache)
    return dict(best, cached=False, trials=trials)
