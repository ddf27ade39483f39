"""Host-side helpers of bench.py that need no GPU: the digest that ties the committed DRAM
traffic record to the tile kernel's code, the lookup that drops the record once that
code changes, and the tile path's time (k_tile plus the centre-split launch).
"""

from __future__ import annotations

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_only_drops_comments_and_keeps_strings():
    src = ('int a = 1; // note\n/* a\n block */ const char *s = "x // y /* z */";\n'
           "char q = '\"';   int  b;\n")
    assert bench.code_only(src) == 'int a = 1; const char *s = "x // y /* z */"; char q = \'"\'; int b;'
    # a comment edit keeps the digest input, a code edit changes it
    assert bench.code_only(src.replace("note", "other note")) == bench.code_only(src)
    assert bench.code_only(src.replace("a = 1", "a = 2")) != bench.code_only(src)


def test_traffic_record_follows_the_kernel_digest(tmp_path, monkeypatch):
    rec = {"dram_bytes_per_launch": 123.0, "source_sha256": bench.kernel_source_digest()}
    path = tmp_path / f"k_tile_{bench.WORKLOAD}.traffic.json"
    path.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_DIR", str(tmp_path))
    assert bench.recorded_traffic() == 123.0
    assert bench.recorded_traffic("uniform_2k_3k") is None
    path.write_text(json.dumps(dict(rec, source_sha256="0" * 64)))
    assert bench.recorded_traffic() is None


def test_tile_path_adds_the_centre_split_launch():
    prof = {"k_tile": (2, 80.0), "k_tile_cs": (2, 20.0), "k_warp_hash": (2, 4.0)}
    assert bench.tile_path_time(prof) == (2, 100.0)
    assert bench.tile_path_time({"k_tile": (3, 30.0)}) == (3, 30.0)
    work = {"k_tile": (10, 1_000_000, 100), "k_warp_hash": (5, 1_000, 10)}
    r = bench.per_kernel_roofline(work, prof, 2, 1000.0)
    # 4 B x 2 visits x 10^6 wedges + 20 B x 100 edges over 50 ms per launch
    assert r["k_tile"]["ms_per_launch"] == 50.0
    assert abs(r["k_tile"]["achieved_gbs"] - 8_002_000 / 0.05 / 1e9) < 1e-12
    assert r["k_warp_hash"]["ms_per_launch"] == 2.0
