"""bench.py's reference arm (the CPU oracle timed on the host cores) prints the JSON line of the
benchmark contract: run here at a small transform size with two worker processes."""
import json

import bench


def test_reference_arm_json_line(monkeypatch, capsys):
    monkeypatch.setattr(bench, "LOGN", 8)
    monkeypatch.setattr(bench, "_cores", lambda: 2)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)

    class Args:
        steps, warmup = 2, 1
    bench.run_reference(Args())
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "NTT/s"
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["vs_baseline"] is None
    assert d["scaling"] == "weak" and d["data"].startswith("synthetic")
    assert "workload" in d["config"] and d["config"]["bits"] == 256
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "NTT/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_are_silent(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class Args:
        steps, warmup = 1, 0
    bench.run_reference(Args())
    assert capsys.readouterr().out == ""
