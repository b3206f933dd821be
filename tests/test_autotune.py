"""Host logic of the segment autotuner: the fastest length wins, lengths the grid
rejects are skipped, the choice is cached by key and reused without timing."""
import json

import pytest

from paper_1910_08324_gb300 import autotune


def test_picks_fastest_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    applied = []
    cost = {16384: 5.0, 32768: 3.0, 65536: 2.5, 131072: 4.0, 262144: 9.0}
    state = {}

    def set_segment(s):
        if s == 262144:
            raise ValueError("too long for this grid")
        state["s"] = s
        applied.append(s)

    def time_ms():
        return cost[state["s"]]

    key = autotune.key_of(1, 4096, 0, [(1024, 2097152), (256, 131072)], boxdit_lmax=16)
    seg, t = autotune.tune_segment(key, set_segment, time_ms, cache_path=path, reps=2)
    assert seg == 65536 and state["s"] == 65536
    assert "262144" not in t and t["65536"] == 2.5
    d = json.load(open(path))
    assert d[key]["segment"] == 65536
    # cached: applied without timing
    applied.clear()
    seg2, _ = autotune.tune_segment(key, set_segment, lambda: pytest.fail("timed again"), cache_path=path)
    assert seg2 == 65536 and applied == [65536]
    # another key is tuned separately; the file keeps both
    key2 = autotune.key_of(2, 8192, 0, [(4096, 1048576)], igrid_depth=1, igrid_layers=4)
    autotune.tune_segment(key2, set_segment, time_ms, cache_path=path, reps=1)
    assert set(json.load(open(path))) == {key, key2}


def test_no_applicable_length_raises():
    def set_segment(s):
        raise ValueError("never")
    with pytest.raises(RuntimeError):
        autotune.tune_segment("k", set_segment, lambda: 1.0)


def test_corrupt_cache_is_ignored(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    seg, _ = autotune.tune_segment("k", lambda s: None, lambda: 1.0, candidates=(32768,), cache_path=str(path))
    assert seg == 32768 and json.load(open(path))["k"]["segment"] == 32768


def test_launch_tuner_searches_both_dimensions_and_caches(tmp_path):
    path = str(tmp_path / "tune.json")
    cost = {(32768, 0): 4.0, (32768, 1): 6.0, (32768, 2): 3.5, (65536, 0): 3.0, (65536, 1): 5.0,
            (65536, 2): 2.0}
    state = {}

    def set_segment(s):
        if s not in (32768, 65536):
            raise ValueError("not for this grid")
        state["s"] = s

    def set_ctas(c):
        if c > 2:
            raise ValueError("more CTAs than fit")
        state["c"] = c

    (seg, c), t = autotune.tune_launch("k", set_segment, set_ctas, lambda: cost[(state["s"], state["c"])],
                                       cache_path=path, reps=2)
    assert (seg, c) == (65536, 2) and (state["s"], state["c"]) == (65536, 2)
    assert t["65536/2"] == 2.0 and "65536/3" not in t and not any(k.startswith("16384/") for k in t)
    d = json.load(open(path))["k"]
    assert (d["segment"], d["ctas_per_sm"]) == (65536, 2)
    state.clear()
    (seg, c), _ = autotune.tune_launch("k", set_segment, set_ctas, lambda: pytest.fail("timed again"),
                                       cache_path=path)
    assert (seg, c) == (65536, 2) and state == {"s": 65536, "c": 2}


def test_general_boxdit_tile_is_tuned_through_the_plan(tmp_path):
    # the general BoxDIT kernel's starts per CTA are what spd_plan_set_segment
    # sets for its plans; the library accepts exactly the tuner's tiles
    spd = pytest.importorskip("paper_1910_08324_gb300")
    plan = spd.spd_plan_create_boxdit([6, 2], 8192, ndm=4, nt=1 << 20)
    cost = {2048: 3.0, 4096: 2.0, 8192: 2.5}
    state = {}

    def set_segment(s):
        spd.spd_plan_set_segment(plan, s)  # raises for a length that is not a tile
        state["s"] = s

    key = autotune.key_of(1, 8192, 0, [(4, 1 << 20)], boxdit_lmax=6)
    seg, t = autotune.tune_segment(key, set_segment, lambda: cost[state["s"]],
                                   candidates=autotune.BOXDIT_GENERAL_TILES + (16384,),
                                   cache_path=str(tmp_path / "t.json"), reps=1)
    assert seg == 4096 and set(t) == {"2048", "4096", "8192"}  # 16384 is not a tile: skipped
