"""The schedule table (host bookkeeping of autotuned schedules) on CPU: JSON round trip, keys,
validation, and which entries `apply` sets, with the library calls replaced by recorders."""
import json

import pytest

from paper_2501_07535_gb300 import moma, schedules


def _cfg(**kw):
    c = {f: 0 for f in schedules.CONFIG_FIELDS}
    c.update(kw)
    return c


def test_round_trip_and_keys(tmp_path):
    t = schedules.Table()
    t.record("ntt_fwd", 1 << 20, 256, False, _cfg(engine=2, tile_log=10, max_logr=5, cta_threads=128), 241.5)
    t.record("mul", 1 << 24, 256, False, _cfg(engine=3, vec_width=1), 454.0)
    t.record("mul", 4096, 256, True, _cfg(engine=4), 12.0)
    # element-wise schedules hold for every length: recorded under n = 0
    assert t.lookup("mul", 17, 256) == _cfg(engine=3, vec_width=1)
    assert t.lookup("mul", 17, 256, full=True) == _cfg(engine=4)
    assert t.lookup("ntt_fwd", 1 << 19, 256) is None
    p = str(tmp_path / "sched.json")
    t.save(p)
    doc = json.load(open(p))
    assert doc["format"] == "moma-schedules" and doc["version"] == 1 and len(doc["entries"]) == 3
    u = schedules.Table.load(p)
    assert u.entries == t.entries


def test_rejects_unknown_content():
    with pytest.raises(ValueError):
        schedules.Table.from_json({"format": "other", "version": 1, "entries": []})
    with pytest.raises(ValueError):
        schedules.Table.from_json({"format": "moma-schedules", "version": 1, "entries": [
            {"op": "mul", "n": 0, "bits": 256, "full": False, "config": {"warp_size": 32}}]})
    with pytest.raises(ValueError):
        schedules.Table().record("fft", 8, 256, False, _cfg())


def test_apply_sets_only_matching_width_and_kind(monkeypatch):
    calls = []
    monkeypatch.setattr(moma, "moma_ctx_set_config", lambda ctx, op, n, **kw: calls.append((ctx, op, n, kw)))
    t = schedules.Table()
    t.record("ntt_fwd", 1 << 12, 256, False, _cfg(tile_log=11), 1.0)
    t.record("ntt_inv", 1 << 12, 256, False, _cfg(tile_log=11), 1.0)
    t.record("axpy", 1 << 20, 256, False, _cfg(engine=2, vec_width=2), 1.0)
    t.record("ntt_fwd", 1 << 12, 384, False, _cfg(tile_log=10), 1.0)
    t.record("mul", 1 << 20, 256, True, _cfg(engine=4), 1.0)
    assert schedules.apply(t, 7, 256) == 3
    assert sorted((op, n) for _, op, n, _ in calls) == [("axpy", 1), ("ntt_fwd", 4096), ("ntt_inv", 4096)]
    assert all(ctx == 7 for ctx, *_ in calls)
    calls.clear()
    assert schedules.apply(t, 9, 256, full=True) == 1
    assert calls == [(9, "mul", 1, _cfg(engine=4))]


def test_tune_records_the_autotuner_choice(monkeypatch):
    monkeypatch.setattr(moma, "moma_autotune", lambda ctx, op, n, count, stream: (_cfg(engine=1, tile_log=9), 3.5))
    t = schedules.Table()
    best = schedules.tune(t, 5, 128, "ntt_fwd", 1 << 14, count=4)
    assert best == _cfg(engine=1, tile_log=9)
    assert t.entries[("ntt_fwd", 1 << 14, 128, False)] == {"config": best, "us": 3.5}
