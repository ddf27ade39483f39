"""Host-side helpers of bench.py that need no GPU: the digest that ties the committed DRAM
traffic record to the tile kernel's code, and the lookup that drops the record once that
code changes.
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
