"""Host logic of the autotuner (no GPU): the candidate set and the tuning cache."""
from paper_1406_1215_gb300 import autotune


def test_candidates_are_distinct_and_start_at_the_defaults():
    for w in (1, 96, 3648):
        c = autotune.default_candidates(w)
        assert c[0] == {}
        assert len(c) == 10
        assert len({tuple(sorted(d.items())) for d in c}) == len(c)
        for d in c:
            assert set(d) <= {"tasks", "block", "blocks_per_sm"}
            assert all(isinstance(v, int) and v > 0 for v in d.values())
            if "block" in d:
                assert d["block"] % 32 == 0 and d["block"] <= 256
    assert autotune.default_candidates(0) == autotune.default_candidates(1)


def test_cache_round_trip_and_damaged_file(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tuning.json"
    monkeypatch.setattr(autotune, "CACHE", str(path))
    assert autotune._load() == {}  # no file yet
    d = {"GB300|152|G1|items2^11": {"knobs": {"tasks": 3648}, "ms": 1.5}}
    autotune._save(d)
    assert autotune._load() == d
    path.write_text("{not json")
    assert autotune._load() == {}  # a damaged cache is ignored, not fatal
