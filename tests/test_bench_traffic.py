"""bench.py's DRAM-traffic bookkeeping (no GPU): an ncu figure is used only while the captured kernel's
source file is unchanged; a workload too large to capture takes a smaller capture's DRAM bytes per
algorithmic byte times its own algorithmic bytes per launch; several forms combine weighed by launches."""
import hashlib
import json

import pytest

import bench


@pytest.fixture
def root(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("// kernel source\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()
    (tmp_path / "profiles").mkdir()
    table = {
        "small": {"a": {"dram_bytes_per_launch": 1000, "source_file": "k.cu", "source_sha256": digest},
                  "stale": {"dram_bytes_per_launch": 5, "source_file": "k.cu", "source_sha256": "0" * 64}},
        "big": {"a": {"scaled_from": "small", "dram_per_alg_byte": 0.75, "source_file": "k.cu",
                      "source_sha256": digest}},
    }
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(table))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def test_captured_and_scaled_entries(root):
    assert bench.stored_traffic("small", "a") == 1000
    assert bench.stored_traffic("small", "a", 4e9) == 1000  # a capture of the workload itself wins
    assert bench.stored_traffic("big", "a", 4e9) == 3_000_000_000
    assert bench.stored_traffic("big", "a") is None  # no algorithmic bytes to scale by
    assert bench.stored_traffic("small", "missing") is None and bench.stored_traffic("other", "a") is None


def test_changed_source_voids_the_entry(root):
    assert bench.stored_traffic("small", "stale") is None
    (root / "k.cu").write_text("// kernel source, edited\n")
    assert bench.stored_traffic("small", "a") is None and bench.stored_traffic("big", "a", 1e9) is None


def test_forms_combine_by_launches():
    roof = {"traffic": None, "forms": {"relax": {"launches": 3, "traffic": 100},
                                       "relax_pull": {"launches": 1, "traffic": 500}}}
    assert bench.combined_traffic(roof)["traffic"] == 200
    roof = {"traffic": None, "forms": {"relax": {"launches": 3, "traffic": 100},
                                       "relax_pull": {"launches": 1, "traffic": None}}}
    assert bench.combined_traffic(roof)["traffic"] is None
    roof = {"traffic": None, "forms": {"relax": {"launches": 0, "traffic": None},
                                       "relax_pull": {"launches": 2, "traffic": 40}}}
    assert bench.combined_traffic(roof)["traffic"] == 40
