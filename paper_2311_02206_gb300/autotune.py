"""Autotuner of the engine's tuning knobs.

The knobs are fields of ``hisa_config`` (include/hisa.h) that change the
speed of a run but never its results:

* ``radix_items``  -- keys per thread of a radix-sort tile (the sort tile):
  the default (24 for 32-bit codes, 12 for 64-bit) or the smaller tile;
* ``load_factor``  -- fill of the open-addressing run index (Section 4.3;
  the paper fixes 0.8, Section 6.2), used where keys are hashed (batched
  and served runs, whose instance ids make the key space too large for a
  direct index);
* ``dense_unit``   -- outer tuples per work unit of the grouped bitmap join
  (the join's work split over CTAs);
* ``pull_ratio``   -- the switch point between push and pull per group.

``tune`` runs a coordinate search: starting from the defaults it tries each
candidate value of one knob with the others held, keeps the fastest, and
moves to the next knob, for a few rounds or until nothing changes.  A trial is
a caller-given function that runs a representative workload through the C-ABI
with a configuration and returns its time.  The best configuration is cached
per shape key (program, domain bits, instance bits, EDB size class) in a JSON
file, so a later session of the same shape starts from it without trials.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import time
from typing import Callable, Dict, Iterable, Optional

DEFAULTS = {"radix_items": 0, "load_factor": 0.8, "dense_unit": 0, "pull_ratio": 4.0}


def knob_candidates(wide: bool, batched: bool) -> Dict[str, list]:
    """Candidate values per knob for codes of 8 bytes (``wide``) or 4, in a
    batched/served run or a single one (pull mode does not run in batches,
    hashed indexes only matter there)."""
    c = {"radix_items": [0, 8 if wide else 16], "dense_unit": [0, 1024, 4096, 16384]}
    if batched:
        c["load_factor"] = [0.5, 0.65, 0.8]
    else:
        c["pull_ratio"] = [2.0, 4.0, 8.0]
    return c


def shape_key(program: str, b: int, inst_bits: int, n_edb: int, mode: str) -> str:
    """Programs, domains and modes tuned alike share a key; EDB sizes are
    bucketed by powers of four."""
    size_class = int(math.log(max(n_edb, 1), 4))
    return f"{program}|b{b}|i{inst_bits}|e4^{size_class}|{mode}"


def default_cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.environ.get("HISA_TUNE_CACHE", os.path.join(base, "hisa", "autotune.json"))


def load_cache(path: Optional[str] = None) -> dict:
    path = path or default_cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: Optional[str] = None) -> None:
    path = path or default_cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(trial: Callable[[dict], float], key: str, candidates: Dict[str, Iterable], rounds: int = 2,
         repeats: int = 1, cache_path: Optional[str] = None, use_cache: bool = True) -> dict:
    """Best configuration for shape ``key``.  ``trial(cfg)`` runs the workload
    with ``cfg`` (DEFAULTS updated by the knobs tried) and returns seconds;
    the median of ``repeats`` calls is compared.  Returns {"config", "trials",
    "seconds", "cached", "times"}."""
    cache = load_cache(cache_path) if use_cache else {}
    if use_cache and key in cache:
        return {"config": dict(cache[key]["config"]), "trials": 0, "seconds": 0.0, "cached": True,
                "times": cache[key].get("times", {})}
    t0 = time.perf_counter()
    timed = {}

    def measure(cfg):
        k = json.dumps(cfg, sort_keys=True)
        if k not in timed:
            timed[k] = statistics.median(trial(dict(cfg)) for _ in range(max(1, repeats)))
        return timed[k]

    best = {k: DEFAULTS[k] for k in candidates}
    best_t = measure(best)
    for _ in range(max(1, rounds)):
        changed = False
        for knob, values in candidates.items():
            for v in values:
                if v == best[knob]:
                    continue
                cfg = dict(best, **{knob: v})
                t = measure(cfg)
                if t < best_t:
                    best, best_t, changed = cfg, t, True
        if not changed:
            break
    out = {"config": best, "trials": len(timed), "seconds": round(time.perf_counter() - t0, 3), "cached": False,
           "times": {k: round(v, 6) for k, v in timed.items()}, "best_seconds": best_t}
    if use_cache:
        cache[key] = {"config": best, "times": out["times"]}
        try:
            save_cache(cache, cache_path)
        except OSError:
            pass
    return out
