"""The benchmark's bookkeeping on CPU: the CSR path's algorithmic bytes for
the record layout, and the DRAM traffic records under profiles/ (returned
only while every source they were captured from is unchanged)."""
import hashlib
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_csr_bytes_per_step_counts_records():
    import bench
    w = {"n": (11, 7), "precision": "fp32"}
    J = 77
    nnz = 3 * 40  # 40 records of 16 B
    want = 40 * 16 + 8.0 * (J + 1) + 4 * J * 11
    assert bench.csr_bytes_per_step(w, nnz) == pytest.approx(want)
    w64 = dict(w, precision="fp64")
    assert bench.csr_bytes_per_step(w64, nnz) == pytest.approx(40 * 32 + 8.0 * (J + 1) + 8 * J * 11)


def test_every_traffic_record_is_read_only_while_current():
    """Each committed record names its kernel, workload and sources under the
    file name bench.py looks up; the bench reports its bytes while the
    digest matches those sources as they stand, and null once one changed
    (a kernel changed since its capture)."""
    import bench
    recs = [f for f in os.listdir(os.path.join(ROOT, "profiles")) if f.endswith(".json")]
    assert recs
    for f in recs:
        d = json.load(open(os.path.join(ROOT, "profiles", f)))
        srcs = d.get("sources") or [d["source"]]
        assert all(os.path.exists(os.path.join(ROOT, s)) for s in srcs), f
        assert d["dram_bytes_per_launch"] > 0, f
        # the file is named <kernel>_<workload>.json, the names bench.py looks up
        wl = d["workload"]
        assert f.endswith(f"_{wl}.json"), f
        name = f[: -len(f"_{wl}.json")]
        current = d["source_sha256"] == bench.sources_sha256(srcs)
        want = d["dram_bytes_per_launch"] if current else None
        assert bench.profile_traffic(name, wl) == want, f
    # the benchmark's own step kernel's record is current
    d = json.load(open(os.path.join(ROOT, "profiles", "k_step2dm_cellular_1025x513.json")))
    assert d["source_sha256"] == bench.sources_sha256(d["sources"])


def test_profile_traffic_is_none_once_a_source_changes(tmp_path, monkeypatch):
    import bench
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    rel = os.path.relpath(str(src), ROOT)
    h = hashlib.sha256(src.read_bytes()).hexdigest()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k_wl.json").write_text(json.dumps({
        "kernel": "k", "workload": "wl", "sources": [rel], "dram_bytes_per_launch": 123,
        "source_sha256": h}))
    monkeypatch.setattr(bench, "PROFILE_DIR", str(prof))
    assert bench.profile_traffic("k", "wl") == 123
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.profile_traffic("k", "wl") is None
    assert bench.profile_traffic("k", "other") is None
