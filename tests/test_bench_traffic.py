"""bench.py reports an ncu traffic figure only while every source file of the kernel still has
the sha256 recorded with the capture (CPU, on a temporary tree)."""
import hashlib
import json
import os

import bench


def _tree(tmp_path, text=b"__global__ void k() {}\n", workload="w"):
    src = tmp_path / "k.cu"
    src.write_bytes(text)
    (tmp_path / "profiles").mkdir()
    rec = {f"k@{workload}": {"dram_bytes_per_launch": 1234.0,
                             "sources": {"k.cu": hashlib.sha256(text).hexdigest()}},
           f"s@{workload}": {"dram_bytes_per_iteration": 10.0,
                             "sources": {"k.cu": hashlib.sha256(text).hexdigest()}}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    return src


def test_traffic_reported_while_sources_match(tmp_path, monkeypatch):
    src = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("k", "w") == 1234.0
    assert bench.measured_traffic("s", "w", iterations=3) == 30.0   # per inner iteration, scaled
    assert bench.measured_traffic("s", "w") is None
    assert bench.measured_traffic("k", "other workload") is None
    assert bench.measured_traffic("missing kernel", "w") is None
    src.write_bytes(b"__global__ void k() { /* changed */ }\n")
    assert bench.measured_traffic("k", "w") is None
    os.remove(src)
    assert bench.measured_traffic("k", "w") is None


def test_committed_record_names_existing_sources():
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for kernel, r in rec.items():
        if kernel.startswith("_"):
            continue
        assert "@" in kernel
        assert r.get("dram_bytes_per_launch", r.get("dram_bytes_per_iteration", 0)) > 0
        for path in r["sources"]:
            assert os.path.exists(os.path.join(bench.ROOT, path)), (kernel, path)
