"""Autotuner for the launch shapes of one solver handle.

It times a few steps for each candidate setting of the knobs exposed by
paces_set_tuning (lanes per row and blocks per SM of the propagator, blocks per
SM of the grid-stride and scan-based kernels, graph replay of whole steps, the
largest load of the hash tables, which sets their size and probe lengths),
always from the same exported state (reloaded with paces_load_state before
every trial), and keeps the fastest setting by coordinate descent.  Choices are
cached in a JSON file keyed by the device name and the model's shape, so later
handles of the same shape start from them.
"""
from __future__ import annotations

import json
import os

from . import binding as B

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paces_tuning.json")


def shape_key(solver, model):
    import torch
    name = torch.cuda.get_device_name(solver.device)
    rows = solver.num_rows()
    scale = len(str(max(rows, 1)))          # decimal order of magnitude of the subspace
    return "%s|N=%d|lat=%d|coup=%d|prec=%d|batch=%d|rows~1e%d" % (
        name, model["n_sites"], model.get("lattice_kind", 0), model.get("coupling_kind", 0),
        model.get("precision", 0), model.get("batch", 1), scale - 1)


def load_cache(path=DEFAULT_CACHE):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache, path=DEFAULT_CACHE):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_steps(solver, state, dt, theta, steps):
    import torch
    solver.load_state(*state)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(solver.stream)
    solver.step(dt, steps, theta)
    e1.record(solver.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def autotune(solver, model, dt, theta, steps=3, cache_path=DEFAULT_CACHE, use_cache=True, log=None):
    """Tune `solver` on its current state; returns (settings, ms per trial)."""
    key = shape_key(solver, model)
    cache = load_cache(cache_path) if cache_path else {}
    if use_cache and key in cache:
        solver.set_tuning(**cache[key]["settings"])
        return cache[key]["settings"], cache[key]["ms"]
    state = solver.state()
    best = solver.tuning()
    best.pop("max_taylor_blocks_per_sm", None)
    best_ms = _time_steps(solver, state, dt, theta, steps)
    lanes = [1, 4, 8]

    def trial(cand):
        try:
            solver.set_tuning(**cand)
        except B.PacesError:
            return None
        return _time_steps(solver, state, dt, theta, steps)

    for knob, values in (("taylor_lanes_per_row", lanes), ("grid_blocks_per_sm", [4, 8, 16]),
                         ("chunk_blocks_per_sm", [2, 4, 6]), ("use_graphs", [0, 1]),
                         ("table_load_pct", [35, 50, 65])):
        for v in values:
            if best.get(knob) == v:
                continue
            cand = dict(best)
            cand[knob] = v
            if knob == "taylor_lanes_per_row":
                solver.set_tuning(**dict(best, taylor_lanes_per_row=v, taylor_blocks_per_sm=1))
                cand["taylor_blocks_per_sm"] = solver.tuning()["max_taylor_blocks_per_sm"]
            ms = trial(cand)
            if log:
                log("%s=%s: %.3f ms" % (knob, v, ms if ms is not None else float("nan")))
            if ms is not None and ms < best_ms:
                best, best_ms = cand, ms
    mx = None
    solver.set_tuning(**best)
    mx = solver.tuning()["max_taylor_blocks_per_sm"]
    for v in sorted({mx, max(1, mx - 1), max(1, mx // 2)}):
        if v == best["taylor_blocks_per_sm"]:
            continue
        ms = trial(dict(best, taylor_blocks_per_sm=v))
        if ms is not None and ms < best_ms:
            best, best_ms = dict(best, taylor_blocks_per_sm=v), ms
    solver.set_tuning(**best)
    solver.load_state(*state)
    if cache_path:
        cache[key] = {"settings": best, "ms": best_ms}
        save_cache(cache, cache_path)
    return best, best_ms
