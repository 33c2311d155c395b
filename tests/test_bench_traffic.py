"""The benchmark's recorded-traffic lookup (CPU only): a per-source DRAM figure is
reported only while every source file it was measured on is unchanged."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _tree(tmp_path, files, entries):
    csrc = tmp_path / "paper_2305_03317_b300" / "csrc"
    csrc.mkdir(parents=True)
    for name, text in files.items():
        (csrc / name).write_text(text)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"entries": entries}))


def _sha(text):
    return hashlib.sha256(text.encode()).hexdigest()


def test_traffic_reported_only_for_unchanged_sources(tmp_path, monkeypatch):
    files = {"a.cu": "kernel A\n", "b.cuh": "shared header\n"}
    entries = {"k|w": {"dram_bytes_per_source": 123.0, "sources": {"a.cu": _sha(files["a.cu"]),
                                                                 "b.cuh": _sha(files["b.cuh"])}}}
    _tree(tmp_path, files, entries)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.committed_traffic("k", "w") == 123.0
    assert bench.committed_traffic("k", "other") is None  # no entry for that workload
    # any listed file changed since the capture: withdrawn
    (tmp_path / "paper_2305_03317_b300" / "csrc" / "b.cuh").write_text("shared header, edited\n")
    assert bench.committed_traffic("k", "w") is None


def test_traffic_missing_or_malformed_record(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.committed_traffic("k", "w") is None  # no record at all
    _tree(tmp_path, {"a.cu": "x"}, {"k|w": {"dram_bytes_per_source": 1.0}})  # no source list
    assert bench.committed_traffic("k", "w") is None
