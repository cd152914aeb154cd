"""Host logic of bench.py (no GPU): the DRAM traffic that a bench line reports
comes from a committed ncu record only while the record matches the kernel
source, the precision, the tile height and the warp roles of the launches."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture
def bench_with_record(tmp_path, monkeypatch):
    import bench
    rec = {
        "source_hash": "h0",
        "precision": "fp32",
        "dram_bytes_per_interior_cell_by_schedule": {"8x1": 95.0, "8x2": 100.0},
        "dram_bytes_per_interior_cell_by_tile_y": {"16": 96.0},
        "refined": {"workload": "w", "schedule": [[16, 304, 1], [8, 912, 2], [8, 912, 2]],
                    "cycle_launches": 7, "cycle_dram_bytes": 700.0},
    }
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k_full_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kfull_source_hash", lambda dtype="f64": "h0")
    return bench


def test_ensemble_traffic_is_keyed_by_tile_height_and_roles(bench_with_record):
    b = bench_with_record
    assert b.kfull_traffic("f32", 10, (8, 912), 2) == 1000.0
    assert b.kfull_traffic("f32", 10, (8, 304), 1) == 950.0
    # the older per-tile-height entries stand for one warp role only
    assert b.kfull_traffic("f32", 10, (16, 912), 1) == 960.0
    assert b.kfull_traffic("f32", 10, (16, 912), 2) is None
    # another precision's launches are not covered
    assert b.kfull_traffic("f64", 10, (8, 912), 1) is None


def test_refined_traffic_needs_the_levels_tile_heights_and_roles(bench_with_record):
    b = bench_with_record
    assert b.refined_kfull_traffic("f32", "w", [[16, 912, 1], [8, 304, 2], [8, 304, 2]]) == 100.0
    # a schedule without its roles is a one-role schedule
    assert b.refined_kfull_traffic("f32", "w", [[16, 304], [8, 912, 2], [8, 912, 2]]) == 100.0
    assert b.refined_kfull_traffic("f32", "w", [[16, 304, 1], [8, 912, 1], [8, 912, 2]]) is None
    assert b.refined_kfull_traffic("f32", "w", [[8, 304, 1], [8, 912, 2], [8, 912, 2]]) is None
    assert b.refined_kfull_traffic("f32", "other", [[16, 304, 1], [8, 912, 2], [8, 912, 2]]) is None


def test_a_changed_source_voids_the_record(bench_with_record, monkeypatch):
    b = bench_with_record
    monkeypatch.setattr(b, "kfull_source_hash", lambda dtype="f64": "h1")
    assert b.kfull_traffic("f32", 10, (8, 912), 2) is None
    assert b.refined_kfull_traffic("f32", "w", [[16, 304, 1], [8, 912, 2], [8, 912, 2]]) is None
