"""Autotuner of the persistent solvers' work schedule.

With the SELL-32 layout each row has one thread, so the schedule knob left is the work-tile size: tiles are
contiguous row ranges (never straddling batch instances) that blocks take in turn. Small tiles balance uneven
batches and instances that converge at different iterations; large tiles mean fewer per-tile partial sums to
reduce at every barrier. The tuner times candidate tile sizes on a live context (rafem_set_schedule rebuilds
only the tile arrays), compares them by solve time per Krylov iteration, keeps the fastest, and caches the choice
in a JSON file keyed by the problem's shape.
"""
from __future__ import annotations

import json
import os

CANDIDATES = (0, 1024, 2048, 4096, 8192, 16384, 32768)


def cache_path() -> str:
    base = os.environ.get("RAFEM_CACHE_DIR") or os.path.join(os.path.expanduser("~"), ".cache", "rafem")
    return os.path.join(base, "autotune.json")


def problem_key(ctx) -> str:
    n_rows, nnz, _ = ctx.pattern_info()
    lay = ctx.layout_info()
    return f"n{n_rows}-nnz{nnz}-inst{ctx.n_inst}-prec{ctx.params.precision}-code{lay['kernel_code']}"


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def autotune_schedule(ctx, candidates=CANDIDATES, steps: int = 2, use_cache: bool = True) -> dict:
    """Pick the tile size with the lowest potential-solve time per Krylov iteration; returns the report.

    The timing runs real time steps on `ctx` (the simulation advances by len(candidates) * steps steps unless the
    choice comes from the cache)."""
    path = cache_path()
    key = problem_key(ctx)
    cache = _load(path) if use_cache else {}
    if key in cache:
        ctx.set_schedule(int(cache[key]["rows_per_tile"]))
        return dict(cache[key], cached=True)
    trials = []
    for rpt in candidates:
        ctx.set_schedule(int(rpt))
        ctx.run(1)  # capture the graph for this schedule outside the measurement
        ctx.set_tracing(True)
        ctx.run(steps)
        tr = ctx.get_trace()
        ctx.set_tracing(False)
        per_iter = tr["ms_solve_V"] / max(1, tr["iters_V"])
        trials.append({"rows_per_tile": ctx.get_schedule()["rows_per_tile"], "request": int(rpt),
                       "ms_per_iteration": per_iter, "ms_solve_V": tr["ms_solve_V"] / steps})
    best = min(trials, key=lambda t: t["ms_per_iteration"])
    ctx.set_schedule(best["rows_per_tile"])
    report = {"rows_per_tile": best["rows_per_tile"], "ms_per_iteration": best["ms_per_iteration"], "trials": trials}
    if use_cache:
        cache[key] = report
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return dict(report, cached=False)
