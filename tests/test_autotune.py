"""Host logic of the launch-knob autotuner: knob bounds, coordinate descent,
the JSON cache.  No GPU: the tuner runs a stand-in workload whose "time" is a
function of the knob values the library holds."""
import json

import pytest


@pytest.fixture()
def at(cr):
    from paper_2005_12692_gb300 import autotune
    autotune.apply(autotune.DEFAULTS)
    yield autotune
    autotune.apply(autotune.DEFAULTS)


def test_defaults_and_bounds(cr, at):
    assert at.current() == at.DEFAULTS
    for name, lo, hi in (("uf_items", 1, 64), ("red_warps", 1, 16), ("uf_compact", 1, 64), ("batch_threads", 0, 3),
                         ("red_budget", 0, 1 << 24)):
        k = at.KNOBS[name]
        for bad in (lo - 1, hi + 1):
            with pytest.raises(cr.CRError) as e:
                cr.cr_tune_set(k, bad)
            assert e.value.code == cr.CR_ERR_INVALID_ARG
            assert at.current()[name] == at.DEFAULTS[name]  # a refused value leaves the knob alone
        cr.cr_tune_set(k, lo)
        assert cr.cr_tune_get(k) == lo
        cr.cr_tune_set(k, hi)
        assert cr.cr_tune_get(k) == hi
    with pytest.raises(cr.CRError):
        cr.cr_tune_set(5, 1)
    with pytest.raises(cr.CRError):
        cr.cr_tune_get(-1)


def test_coordinate_descent_picks_the_fastest(cr, at):
    # stand-in cost: a bowl in uf_items (best 4) plus a term in uf_compact (best 16)
    calls = []

    def run():
        calls.append(at.current())

    def timer(fn):
        fn()
        v = at.current()
        return abs(v["uf_items"] - 4) * 1.0 + abs(v["uf_compact"] - 16) * 0.5 + 10.0

    res = at.autotune(run, {"uf_items": [2, 4, 8, 16], "uf_compact": [1, 4, 16, 64]}, warmup=1, repeats=3,
                      timer=timer)
    assert res.best == {"uf_items": 4, "red_warps": 16, "uf_compact": 16, "batch_threads": 2, "red_budget": 1024}
    assert at.current() == res.best  # left set in the library
    # every candidate was timed once in the table; the second knob was timed with the first at its best
    assert [(k, v) for k, v, _ in res.table] == [("uf_items", 2), ("uf_items", 4), ("uf_items", 8),
                                                 ("uf_items", 16), ("uf_compact", 1), ("uf_compact", 4),
                                                 ("uf_compact", 16), ("uf_compact", 64)]
    assert all(c["uf_items"] == 4 for c in calls if c["uf_compact"] != 1)
    assert len(calls) == 8 * (1 + 3)  # warm-up + timed calls per candidate
    d = res.as_dict()
    assert d["best"]["uf_items"] == 4 and len(d["table"]) == 8


def test_ties_keep_the_earlier_candidate_and_bad_input_raises(cr, at):
    res = at.autotune(lambda: None, {"red_warps": [16, 8, 4]}, warmup=0, repeats=1, timer=lambda fn: 1.0)
    assert res.best["red_warps"] == 16
    with pytest.raises(KeyError):
        at.autotune(lambda: None, {"nonsense": [1]}, timer=lambda fn: 1.0)
    with pytest.raises(ValueError):
        at.autotune(lambda: None, {"uf_items": [8]}, repeats=0, timer=lambda fn: 1.0)
    with pytest.raises(cr.CRError):
        at.autotune(lambda: None, {"uf_items": [0]}, timer=lambda fn: 1.0)


def test_cache_round_trip(at, tmp_path):
    path = str(tmp_path / "tuning.json")
    assert at.load(path, "dev|grf1024") is None
    at.save(path, "dev|grf1024", {"uf_items": 4, "uf_compact": 16})
    at.save(path, "dev|batch4096", {"uf_compact": 2})
    assert at.load(path, "dev|grf1024") == {"uf_items": 4, "uf_compact": 16}
    assert at.load(path, "dev|batch4096") == {"uf_compact": 2}
    with open(path) as f:
        assert set(json.load(f)) == {"dev|grf1024", "dev|batch4096"}
    at.apply(at.load(path, "dev|grf1024"))
    assert at.current()["uf_items"] == 4
