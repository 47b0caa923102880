"""Host logic of the launch-shape autotuner (no GPU needed)."""
from paper_2602_11734_gb300 import tune


def test_candidate_shapes_stay_within_one_wave():
    shapes = tune.candidate_shapes(152)
    assert (456, 1) in shapes and (152, 8) in shapes
    assert all(b <= 3 * 152 and b % 152 == 0 for b, _ in shapes)
    assert all(1 <= t <= 16 for _, t in shapes)
    assert len(shapes) == len(set(shapes)) == len(tune.BLOCKS_PER_SM) * len(tune.TILES)


def test_pick_best_sums_points_and_breaks_ties_deterministically():
    timings = {(456, 1): [1.0, 2.0, 3.0], (304, 2): [1.5, 1.5, 2.0], (152, 4): [5.0, 0.1, 0.1]}
    assert tune.pick_best(timings) == (304, 2)
    tied = {(456, 2): [2.0], (304, 4): [2.0], (304, 1): [2.0]}
    assert tune.pick_best(tied) == (304, 1)


def test_cache_round_trip(tmp_path, monkeypatch):
    monkeypatch.setenv("QSGS_TUNE_CACHE", str(tmp_path / "sub" / "tune.json"))
    tune._store("k1", {"blocks": 304, "tile": 2})
    tune._store("k2", {"blocks": 456, "tile": 1})
    cache = tune._load_cache()
    assert cache["k1"] == {"blocks": 304, "tile": 2} and cache["k2"]["blocks"] == 456
