"""Autotuner of the contraction kernels' launch grids for batches of independent problems.

Each hour-angle handle runs its forward and adjoint contractions on a grid of CTAs
(fm_set_launch_grids; one CTA per SM by default).  In the batched schedule of independent
HMC chains the problems run as concurrent branches of one CUDA graph, so a problem that
keeps every SM for itself serialises the batch, while one that takes fewer CTAs than it can
use runs longer.  The tuner

1. times, per problem shape (antennas, fringe groups, channels, declinations, hour-angle
   cells, LSTs, precision), one chi^2 + gradient evaluation at each candidate grid, standalone,
   with CUDA events (`measure`), and caches the times in a JSON file keyed by the shape, so a
   shape seen before is not timed again;
2. gives each problem the fewest CTAs whose time is within a factor `slack` of the shape's
   best (`choose`);
3. `tune_batch` tries several slacks on the batch itself (one graph per try) and keeps the
   one with the shortest step.

All of it is host-side scheduling: the kernels and their arithmetic are unchanged (a grid
change only regroups the forward's partial sums).
"""
from __future__ import annotations

import json
import os
import time

import torch

from . import fm

CANDIDATES = (8, 16, 19, 38, 76, 152)


def default_cache_path() -> str:
    base = os.environ.get("FM_TUNE_CACHE")
    if base:
        return base
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2504_07090_gb300", "launch_grids.json")


def shape_key(model: "fm.ForwardModel") -> str:
    info = model.contraction_info()
    p = model.prob
    return (f"A{p.n_ant}-U{info['fringes']}-F{p.n_freq}-D{p.n_dec}-R{p.n_ra}-H{info['hour_angle_cells']}"
            f"-T{p.n_lst}-k{info['lst_step_cells']}-{model.precision}")


def load_cache(path: str) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: dict) -> None:
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def measure(model: "fm.ForwardModel", theta: torch.Tensor, candidates=CANDIDATES, reps: int = 5) -> dict:
    """Milliseconds per chi^2 + gradient evaluation of `model` at each candidate grid (the same
    count of CTAs for the forward and the adjoint), after one untimed evaluation per grid."""
    sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    st = torch.cuda.current_stream()
    scal = torch.empty(2, dtype=torch.float64, device="cuda")
    grad = torch.empty_like(theta)
    out = {}
    for g in sorted({min(int(c), sm) for c in candidates}):
        model.set_launch_grids(g, g)
        model.chi2_grad(theta, grad, scal)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(reps):
            model.chi2_grad(theta, grad, scal)
        b.record(st)
        torch.cuda.synchronize()
        out[str(g)] = a.elapsed_time(b) / reps
    model.set_launch_grids(0, 0)
    return out


def choose(times: dict, slack: float) -> int:
    """The fewest CTAs whose time is within `slack` times the best."""
    best = min(times.values())
    ok = [int(g) for g, t in times.items() if t <= slack * best]
    return min(ok)


def shape_times(models, thetas, cache_path: str | None = None, candidates=CANDIDATES, reps: int = 5):
    """Per-model timing tables, from the cache where the shape was seen before.
    Returns (tables, n_timed): tables[k] is None for a model without the hour-angle form."""
    path = cache_path or default_cache_path()
    cache = load_cache(path)
    tables, timed = [], 0
    for m, th in zip(models, thetas):
        if m.contraction_info()["form"] != "hour_angle":
            tables.append(None)
            continue
        key = shape_key(m)
        if key not in cache:
            cache[key] = measure(m, th, candidates, reps)
            timed += 1
        tables.append(cache[key])
    if timed:
        save_cache(path, cache)
    return tables, timed


def apply(models, tables, slack: float) -> list:
    """Set every hour-angle model's grids from its table; returns the chosen CTA counts."""
    chosen = []
    for m, tab in zip(models, tables):
        if tab is None:
            chosen.append(None)
            continue
        g = choose(tab, slack)
        m.set_launch_grids(g, g)
        chosen.append(g)
    return chosen


def tune_batch(models, thetas, run_step, slacks=(1.0, 1.25, 1.5, 2.0, 3.0), cache_path: str | None = None,
               candidates=CANDIDATES):
    """Pick the slack whose grids give the shortest batch step.  run_step() must build the batch
    for the models' current grids, run it and return its milliseconds per step.  Returns a
    report: the slack chosen, the step time of each slack and of the default grids, and the
    number of shapes that had to be timed."""
    t0 = time.perf_counter()
    tables, timed = shape_times(models, thetas, cache_path, candidates)
    for m, tab in zip(models, tables):
        if tab is not None:
            m.set_launch_grids(0, 0)
    default_ms = run_step()
    steps = {}
    for s in slacks:
        apply(models, tables, s)
        steps[str(s)] = run_step()
    best = min(steps, key=steps.get)
    if steps[best] >= default_ms:
        for m, tab in zip(models, tables):
            if tab is not None:
                m.set_launch_grids(0, 0)
        chosen = "default"
    else:
        apply(models, tables, float(best))
        chosen = float(best)
    grids = [m.launch_grids()[0] if tab is not None else None for m, tab in zip(models, tables)]
    return {"slack": chosen, "ms_per_step": {"default": default_ms, **steps}, "shapes_timed": timed,
            "shapes": len({shape_key(m) for m, tab in zip(models, tables) if tab is not None}),
            "grids": {"min": min(g for g in grids if g), "max": max(g for g in grids if g)},
            "tuning_s": time.perf_counter() - t0}
