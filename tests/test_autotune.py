"""The autotuner's search and cache (paper_2311_02206_gb300.autotune) with a
synthetic trial function: no GPU."""
import json

from paper_2311_02206_gb300 import autotune


def _trial_factory(optimum, calls):
    def trial(cfg):
        calls.append(dict(cfg))
        # separable cost with its minimum at `optimum`
        cost = 1.0
        for k, v in optimum.items():
            cost += abs(float(cfg[k]) - float(v)) / (1.0 + abs(float(v)))
        return cost
    return trial


def test_coordinate_search_finds_the_optimum(tmp_path):
    cands = {"radix_items": [0, 16], "dense_unit": [0, 1024, 4096, 16384], "pull_ratio": [2.0, 4.0, 8.0]}
    optimum = {"radix_items": 16, "dense_unit": 4096, "pull_ratio": 8.0}
    calls = []
    res = autotune.tune(_trial_factory(optimum, calls), "k", cands, cache_path=str(tmp_path / "c.json"))
    assert res["config"] == optimum
    assert not res["cached"] and res["trials"] == len(calls)
    assert res["trials"] <= 1 + 2 * sum(len(v) for v in cands.values())


def test_cache_round_trip_and_keys(tmp_path):
    path = str(tmp_path / "c.json")
    cands = {"load_factor": [0.5, 0.65, 0.8]}
    calls = []
    first = autotune.tune(_trial_factory({"load_factor": 0.65}, calls), "shape", cands, cache_path=path)
    n = len(calls)
    again = autotune.tune(_trial_factory({"load_factor": 0.65}, calls), "shape", cands, cache_path=path)
    assert again["cached"] and again["trials"] == 0 and len(calls) == n
    assert again["config"] == first["config"] == {"load_factor": 0.65}
    assert json.load(open(path))["shape"]["config"] == {"load_factor": 0.65}
    other = autotune.tune(_trial_factory({"load_factor": 0.5}, calls), "other", cands, cache_path=path)
    assert not other["cached"] and other["config"] == {"load_factor": 0.5}


def test_shape_keys_and_candidates():
    a = autotune.shape_key("reach", 13, 12, 5000, "served")
    b = autotune.shape_key("reach", 13, 12, 6000, "served")
    c = autotune.shape_key("reach", 13, 12, 50000, "served")
    assert a == b != c
    assert autotune.knob_candidates(True, True)["radix_items"] == [0, 8]
    assert "pull_ratio" in autotune.knob_candidates(False, False)
    assert "load_factor" in autotune.knob_candidates(False, True)
