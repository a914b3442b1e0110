"""The tuner's table on the CPU: ranges cover every N once, the JSON round trip
keeps the knobs."""
from paper_1208_2675_gb300 import tuner


def test_ranges_cover_every_size_once():
    table = {100: {"knobs": {"tier": 0}}, 60: {"knobs": {"tier": 3}},
             1024: {"knobs": {"t3_grid": 76}}}
    r = tuner.ranges(table)
    assert [x[0] for x in r] == [2, 81, 563]
    assert [x[1] for x in r] == [80, 562, 2 ** 31 - 1]
    for n in [2, 60, 80, 81, 100, 562, 563, 5000]:
        hits = [k for lo, hi, k in r if lo <= n <= hi]
        assert len(hits) == 1
    assert r[0][2] == {"tier": 3}


def test_json_round_trip(tmp_path):
    table = {256: {"knobs": {"tier": 0, "hybrid_rate": 0.001}, "seconds": 1.5, "iters": 10}}
    path = str(tmp_path / "t.json")
    tuner.save(path, table, {"x": 1})
    assert tuner.load(path) == table


def test_trial_length_is_bounded():
    for N in (2, 12, 100, 1024, 3000):
        assert 10 ** 6 <= tuner.tuning_iters(N) <= 2 * 10 ** 7
