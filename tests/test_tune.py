"""The launch-shape tuning table (host only): lookup order, validation, the
JSON cache reader, and that the autotuner's knob list matches the library's."""
import json
import math

import pytest

from paper_2201_00730_gb300 import autotune as A
from paper_2201_00730_gb300 import uot as U


@pytest.fixture(autouse=True)
def clean_table():
    U.tune_clear()
    yield
    U.tune_clear()


def test_bucket_is_floor_log2():
    for e in (2, 3, 4, 1000, 20000 * 20000, 262144 ** 2, 2 ** 40 - 1, 2 ** 40):
        assert U.tune_bucket(e) == math.floor(math.log2(e))
    assert U.tune_bucket(1) == 0 and U.tune_bucket(0) == 0


def test_most_specific_entry_wins():
    b = U.tune_bucket(20000 * 20000)
    assert U.tune_get("tile.rows", 3, 20000 * 20000) == 0
    U.tune_set("tile.rows", 4)
    U.tune_set("tile.rows", 2, dim=3)
    U.tune_set("tile.rows", 4, dim=3, bucket=b)
    U.tune_set("tile.rows", 2, bucket=b + 1)
    assert U.tune_get("tile.rows", 3, 20000 * 20000) == 4       # (dim, bucket)
    assert U.tune_get("tile.rows", 3, 2 * 20000 * 20000) == 2   # (dim, any) before (any, bucket)
    assert U.tune_get("tile.rows", 2, 2 * 20000 * 20000) == 2   # (any, bucket)
    assert U.tune_get("tile.rows", 2, 100) == 4                 # (any, any)
    assert U.tune_get("tile.rows", 3, 0) == 2                   # no size: bucket entries skipped
    U.tune_set("tile.rows", 0, dim=3)                           # 0 clears
    assert U.tune_get("tile.rows", 3, 2 * 20000 * 20000) == 2   # now (any, bucket)
    U.tune_clear()
    assert U.tune_get("tile.rows", 3, 20000 * 20000) == 0


def test_only_allowed_values_and_known_knobs():
    for knob, vals in A.KNOBS.items():
        for v in vals:
            U.tune_set(knob, v, dim=2, bucket=20)
            assert U.tune_get(knob, 2, 2 ** 20) == v
        for bad in (-1, 3 if knob != "points.resident" and knob != "batch.ctas_per_sm" else 5, 7, 16384):
            if bad in vals:
                continue
            with pytest.raises(U.UOTError):
                U.tune_set(knob, bad)
    with pytest.raises(U.UOTError):
        U.tune_set("tile.unknown", 2)
    with pytest.raises(U.UOTError):
        U.tune_set("tile.rows", 2, dim=65)
    with pytest.raises(U.UOTError):
        U.tune_set("tile.rows", 2, bucket=200)


def test_cache_round_trip(tmp_path):
    cache = {"device": "any", "sm_count": 1, "created": "x", "entries": [
        {"knob": "tile.rows", "dim": 3, "bucket": 28, "value": 2},
        {"knob": "dense.col_ctas", "dim": -1, "bucket": -1, "value": 8},
        {"knob": "batch.ctas_per_sm", "dim": -1, "bucket": -1, "value": 1, "note": {"a": [1, 2]}}]}
    p = tmp_path / "tune.json"
    p.write_text(json.dumps(cache, indent=2))
    U.tune_load(str(p))
    assert U.tune_get("tile.rows", 3, 20000 * 20000) == 2
    assert U.tune_get("tile.rows", 3, 10 ** 6) == 0
    assert U.tune_get("dense.col_ctas", -1, 10 ** 6) == 8
    assert U.tune_get("batch.ctas_per_sm", -1, 0) == 1
    assert A.load(str(p), check_device=False)


def test_bad_cache_changes_nothing(tmp_path):
    U.tune_set("tile.cta_cost", 25)
    for text in ('{"entries": [{"knob": "tile.rows", "dim": 3, "bucket": 28, "value": 3}]}',
                 '{"entries": [{"knob": "tile.rows", "dim": 3, "bucket": 28, "value": 2}, {"knob": "x", "value": 1}]}',
                 '{"entries": [', "not json"):
        p = tmp_path / "bad.json"
        p.write_text(text)
        with pytest.raises(U.UOTError):
            U.tune_load(str(p))
        assert U.tune_get("tile.rows", 3, 20000 * 20000) == 0
        assert U.tune_get("tile.cta_cost", 3, 20000 * 20000) == 25
    with pytest.raises(U.UOTError):
        U.tune_load(str(tmp_path / "missing.json"))
