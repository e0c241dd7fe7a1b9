"""Host logic of the launch autotuner: cache keys, candidate sets, selection and the JSON
cache (no GPU)."""
import json

from paper_2409_07392_gb300 import autotune as at


def test_shape_key_rounds_n_to_a_power_of_two():
    assert at.shape_key("mixed_fast", 1_000_000, 64, 1000, 16) == "mixed_fast:n2^20:d64:c1000:s16"
    assert at.shape_key("mixed", 3000, 16, 10, 8) == at.shape_key("mixed", 3500, 16, 10, 8)
    assert at.shape_key("mixed", 3000, 16, 10, 8) != at.shape_key("mixed", 12000, 16, 10, 8)


def test_candidates_surround_the_rule_and_stay_positive():
    cands = at.candidates({"dterm_splits": 38, "bsum_splits": 19})
    ds = {c["dterm_splits"] for c in cands}
    bs = {c["bsum_splits"] for c in cands}
    assert 38 in ds and 19 in bs and min(ds) == 19 and max(ds) == 76
    assert all(c["sm_budget"] == 0 for c in cands)
    tiny = at.candidates({"dterm_splits": 1, "bsum_splits": 0})
    assert all(c["dterm_splits"] >= 1 and c["bsum_splits"] >= 1 for c in tiny)


def test_pick_best_prefers_the_earlier_on_ties():
    a, b = {"dterm_splits": 0}, {"dterm_splits": 5}
    assert at.pick_best([(a, 2.0), (b, 2.0)]) == (a, 2.0)
    assert at.pick_best([(a, 2.0), (b, 1.5)]) == (b, 1.5)


def test_cache_round_trip_and_validation(tmp_path):
    path = tmp_path / "sub" / "tune.json"
    c = at.TuneCache(str(path))
    assert c.get("k") is None
    c.put("k", {"dterm_splits": 4, "bsum_splits": 2, "sm_budget": 0, "ms": 1.0})
    c2 = at.TuneCache(str(path))
    assert c2.get("k") == {"dterm_splits": 4, "bsum_splits": 2, "sm_budget": 0}
    # malformed entries and files are ignored, not trusted
    path.write_text(json.dumps({"k": {"dterm_splits": -1, "bsum_splits": 2, "sm_budget": 0}}))
    assert at.TuneCache(str(path)).get("k") is None
    path.write_text("not json")
    assert at.TuneCache(str(path)).data == {}


def test_apply_cached_sets_the_stored_tuning(tmp_path):
    class FakeProblem:
        precision, n, d, c = "mixed", 4096, 32, 10

        def __init__(self):
            self.set = None

        def set_tuning(self, **kw):
            self.set = kw

    cache = at.TuneCache(str(tmp_path / "t.json"))
    p = FakeProblem()
    assert not at.apply_cached(p, 8, cache)
    cache.put(at.shape_key("mixed", 4096, 32, 10, 8),
              {"dterm_splits": 3, "bsum_splits": 7, "sm_budget": 76})
    assert at.apply_cached(p, 8, cache)
    assert p.set == {"dterm_splits": 3, "bsum_splits": 7, "sm_budget": 76}
