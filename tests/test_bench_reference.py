"""The reference arm of bench.py (the FP64 CPU oracle, no GPU): one JSON line with
the contract's keys, on the 32^3 ridge workload."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.main(["--impl", "reference", "--workload", "ridge", "--steps", "2", "--warmup", "1"]) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"]


def test_reference_arm_sgs_workload(monkeypatch, capsys):
    """The reference arm of the SGS workload: the oracle's Smagorinsky stress, wall stress and force
    on the cube array, reported under the GPU arm's metric, on one core."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.main(["--impl", "reference", "--workload", "sgs", "--steps", "1", "--warmup", "0"]) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC_SGS
    assert d["value"] > 0 and d["cpu_baseline"]["cores"] == 1
    assert "SGS stress" in d["cpu_baseline"]["sample"]
    assert d["config"]["nodes"] == 256 * 128 * 128


def test_reference_arm_sdf_workload(monkeypatch, capsys):
    """The reference arm of the height-field distance: the oracle's brute force on
    near-surface nodes of the hill, under the GPU arm's metric, on one core."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.main(["--impl", "reference", "--workload", "sdf", "--steps", "1", "--warmup", "0"]) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC_SDF
    assert d["value"] > 0 and d["cpu_baseline"]["cores"] == 1 and d["dtype"] == "f64"
    assert d["e2e"]["value"] == d["value"]


def test_reference_arm_ensemble_workload(monkeypatch, capsys):
    """The reference arm of the default (batched ensemble) workload on a few members:
    the oracle's wall stress + force over every member, under the GPU arm's metric
    and workload name."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.main(["--impl", "reference", "--members", "3", "--steps", "1", "--warmup", "0"]) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["config"]["members"] == 3 and d["config"]["workload"].startswith("ensemble of 3")
    assert d["value"] > 0 and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"]
