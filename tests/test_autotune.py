"""Host logic of the option autotuner (search, objective bookkeeping, cache), with a
deterministic stand-in for the GPU measurement."""
import json

import numpy as np

from paper_2607_07485_b300 import autotune as AT


def _cost(opts):
    # separable stand-in with its minimum away from the defaults
    return (abs(opts["large_dense"] - 4096) / 1024 + abs(opts["split_sweep"] - 64) / 64
            + (0.5 if opts["sweep_block"] == 64 else 0.0))


def test_tune_finds_the_minimum_and_measures_each_configuration_once():
    calls = []

    def measure(o):
        calls.append(tuple(sorted(o.items())))
        return _cost(o)

    best, table = AT.tune(measure)
    assert best == {"large_dense": 4096, "split_sweep": 64, "sweep_block": 32}
    assert len(calls) == len(set(calls)) == len(table)
    assert min(table.values()) == _cost(best)


def test_tune_keeps_the_defaults_when_nothing_is_faster():
    best, _ = AT.tune(lambda o: 1.0)
    assert best == AT.DEFAULTS


def test_autotune_cache_round_trip(tmp_path):
    cache = str(tmp_path / "tune.json")
    dofs = np.zeros((10, 4), np.int32)
    n_calls = [0]

    def measure(o):
        n_calls[0] += 1
        return _cost(o)

    best = AT.autotune(100, dofs, None, cache_file=cache, measure=measure, device="dev0")
    first = n_calls[0]
    assert first > 0 and best["large_dense"] == 4096
    again = AT.autotune(100, dofs, None, cache_file=cache, measure=measure, device="dev0")
    assert again == best and n_calls[0] == first          # served from the cache
    other = AT.autotune(100, dofs, None, cache_file=cache, measure=measure, device="dev1")
    assert other == best and n_calls[0] == 2 * first      # another device is tuned afresh
    data = json.load(open(cache))
    assert len(data) == 2 and all("measured" in v for v in data.values())
