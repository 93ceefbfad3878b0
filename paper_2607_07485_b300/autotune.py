"""Autotuner for the library's tile-shape and kernel-variant options.

Three options decide tile shapes and which kernel variant runs:
  large_dense  local eigenproblem order above which the tridiagonalisation runs on many CTAs
               per matrix instead of one (set-up);
  split_sweep  overlap size above which a Schwarz colour uses the blocked many-CTA triangular
               solves instead of one CTA per subdomain (every V-cycle);
  sweep_block  rows per diagonal block of the blocked triangular solves (set-up and V-cycle).

The tuner measures candidates on the caller's problem, or on a smaller one of the same element
type when a full set-up per candidate is too costly.  It runs coordinate descent from the
library defaults, and each distinct configuration is measured once.  The objective is the
set-up time plus `cycles` V-cycle applications, timed with CUDA events on the current stream.
Results are cached in a JSON file keyed by the device name and a problem signature, so a later
call with the same key returns the tuned options without measuring.

    from paper_2607_07485_b300.autotune import autotune
    opts = autotune(n, elem_dofs, elem_mats, coef, cache_file="lsamg_tune.json")
    amg = Lsamg(n, elem_dofs, elem_mats, coef, **opts)
"""
from __future__ import annotations

import json
import os

DEFAULTS = {"large_dense": 2048, "split_sweep": 128, "sweep_block": 64}
SPACE = {"large_dense": (1024, 2048, 4096), "split_sweep": (64, 128, 512), "sweep_block": (32, 64)}


def problem_key(device: str, n: int, n_elems: int, n_T: int, extra: dict | None = None) -> str:
    """Cache key: the device and the problem's size signature (plus the fixed options)."""
    tail = "" if not extra else "|" + ",".join(f"{k}={extra[k]}" for k in sorted(extra))
    return f"{device}|n={n}|ne={n_elems}|nT={n_T}{tail}"


def tune(measure, space=SPACE, start=None, sweeps=1):
    """Coordinate descent over `space` from `start` (default: the library defaults).
    measure(opts) -> seconds, lower is better; each distinct configuration is measured once.
    Returns (best options, {configuration tuple: seconds})."""
    best = dict(DEFAULTS if start is None else start)
    table = {}

    def cost(opts):
        key = tuple(sorted(opts.items()))
        if key not in table:
            table[key] = float(measure(dict(opts)))
        return table[key]

    best_t = cost(best)
    for _ in range(sweeps):
        for name, values in space.items():
            for v in values:
                cand = dict(best, **{name: v})
                t = cost(cand)
                if t < best_t:
                    best, best_t = cand, t
    return best, table


def gpu_measure(n, elem_dofs, elem_mats, coef=None, cycles=20, reps=3, base_opts=None):
    """measure(opts) for `tune`: set-up seconds of a handle built with `opts` (from its own
    statistics) plus `cycles` times the median of `reps` timed V-cycle applications."""
    import torch

    from .lsamg import Lsamg

    def measure(opts):
        amg = Lsamg(n, elem_dofs, elem_mats, coef, **dict(base_opts or {}, **opts))
        try:
            setup_s = amg.stats()["setup_seconds"]
            r = torch.ones(n, dtype=torch.float64, device=elem_dofs.device)
            amg.apply(r)                       # warm-up
            times = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                amg.apply(r)
                e1.record()
                e1.synchronize()
                times.append(e0.elapsed_time(e1) / 1000.0)
            times.sort()
            return setup_s + cycles * times[len(times) // 2]
        finally:
            amg.close()

    return measure


def autotune(n, elem_dofs, elem_mats, coef=None, cache_file=None, cycles=20, space=SPACE, base_opts=None,
             measure=None, device=None):
    """Tuned {large_dense, split_sweep, sweep_block} for this problem (see the module docstring).
    `measure` and `device` default to the GPU measurement and the current device's name."""
    if device is None:
        import torch
        device = torch.cuda.get_device_name()
    key = problem_key(device, int(n), int(elem_dofs.shape[0]), int(elem_dofs.shape[1]), base_opts)
    cache = {}
    if cache_file and os.path.exists(cache_file):
        with open(cache_file) as f:
            cache = json.load(f)
        if key in cache:
            return dict(cache[key]["options"])
    if measure is None:
        measure = gpu_measure(n, elem_dofs, elem_mats, coef, cycles=cycles, base_opts=base_opts)
    best, table = tune(measure, space)
    if cache_file:
        cache[key] = dict(options=best, measured={",".join(f"{k}={v}" for k, v in cfg): t
                                                  for cfg, t in table.items()})
        tmp = cache_file + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_file)
    return best
