"""bench.py's roofline inputs on the CPU: DRAM traffic is taken from the committed ncu summary only
when that summary was measured on the current source of the kernel and on the line's own workload
(or on a smaller case of it, scaled by the algorithmic bytes), and the byte models follow their
per-unit figures."""
import hashlib
import json
import os

import bench


def _tree(tmp_path, source_text: bytes, entry: dict):
    csrc = tmp_path / "paper_2010_10055_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_bytes(source_text)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps({"kern": entry}))


def _entry(source_text: bytes, **kw):
    e = {"dram_bytes_per_launch": 1000.0, "source": "k.cu",
         "source_sha256_16": hashlib.sha256(source_text).hexdigest()[:16]}
    e.update(kw)
    return e


def test_traffic_of_the_same_workload_and_source(tmp_path, monkeypatch):
    src = b"__global__ void k() {}\n"
    _tree(tmp_path, src, _entry(src, workload="w"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("kern", "w") == 1000.0
    assert bench.measured_traffic("kern", "other") is None  # another read set: not this line's traffic
    assert bench.measured_traffic("missing", "w") is None


def test_traffic_of_a_smaller_case_is_scaled(tmp_path, monkeypatch):
    src = b"__global__ void k() {}\n"
    _tree(tmp_path, src, _entry(src, workload="w@0.05", small_case_of="w", algorithmic_bytes_per_launch=500.0))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("kern", "w", launch_bytes=2000.0) == 4000.0
    assert bench.measured_traffic("kern", "w") is None  # no algorithmic bytes to scale by
    assert bench.measured_traffic("kern", "v", launch_bytes=2000.0) is None


def test_traffic_of_changed_source_is_stale(tmp_path, monkeypatch):
    src = b"__global__ void k() {}\n"
    _tree(tmp_path, src, _entry(src, workload="w"))
    (tmp_path / "paper_2010_10055_gb300" / "csrc" / "k.cu").write_bytes(src + b"// changed\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("kern", "w") is None


def test_committed_summary_names_existing_sources():
    t = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for name, e in t.items():
        assert os.path.exists(os.path.join(bench.ROOT, "paper_2010_10055_gb300", "csrc", e["source"])), name
        assert e["dram_bytes_per_launch"] > 0 and e["algorithmic_bytes_per_launch"] > 0


def test_byte_models():
    k = {"candidates": 100, "nnz": 60, "m": 20, "sort_passes": 4, "a_sort_passes": 3, "sort_key_bytes": 8,
         "sort_val_bytes": 0, "bloom_bins": 0}
    sz = dict(n=10, total=1000, windows=900, nnzA=60, products=200, products_half=70, upper=True, nnzC=40, S=2,
              nnzR=30, tr_products=90, rounds=2, kstats=k, direct_seg=True)
    # every pass reads and writes each key; the sort of A moves (4-byte key, 8-byte value) pairs
    assert bench.algorithmic_bytes("radix_onesweep", sz) == 2 * 4 * 100 * 8 + 2 * 3 * 60 * 12
    # upper triangle: half the off-diagonal products and half of C (8 + 8 S bytes an entry)
    assert bench.algorithmic_bytes("spgemm_numeric", sz) == 8 * 60 + 8 * 70 + (8 + 16) * 40 / 2 + 8 * 11
    assert bench.algorithmic_bytes("seg_mark", sz) == 8.25 * 100
    assert bench.algorithmic_bytes("emit_at", sz) == 8.25 * 100 + 20 * 60 + 16 * 20
    assert bench.algorithmic_bytes("seg_mark", dict(sz, direct_seg=False)) is None
    assert bench.algorithmic_bytes("pack", sz) == 5.25 * 1000
    assert bench.algorithmic_bytes("tr_minplus_mark", sz) == (9 * 30 + 9 * 90 + 30 + 8 * 10) * 2
