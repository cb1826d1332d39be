"""Host logic of bench.py that needs no GPU: the committed traffic record's
parser and its source guard, and the reference arm's JSON line (the oracle
timed on a bounded sample) on a tiny workload."""
import argparse
import hashlib
import io
import json
import os
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import rime_synth  # noqa: E402


def _src_md5():
    with open(os.path.join(ROOT, "paper_1501_07719_gb300", "csrc", "rime_fused.cu"), "rb") as f:
        return hashlib.md5(f.read()).hexdigest()


def test_traffic_record_is_read_only_for_the_captured_source(tmp_path, monkeypatch):
    rec = tmp_path / "traffic.txt"
    monkeypatch.setattr(bench, "TRAFFIC_RECORD", str(rec))
    rec.write_text(f"# comment\ntraffic_bytes_per_launch: 123456\nsource_md5: {_src_md5()[:12]} (note)\n")
    assert bench.profiled_traffic() == 123456
    rec.write_text("traffic_bytes_per_launch: 123456\nsource_md5: 000000000000\n")
    assert bench.profiled_traffic() is None          # the kernel changed since the capture
    rec.write_text(f"source_md5: {_src_md5()[:12]}\n")
    assert bench.profiled_traffic() is None          # no traffic key
    rec.unlink()
    assert bench.profiled_traffic() is None          # no record


def test_committed_traffic_record_parses():
    """The committed record has both keys (its md5 may lag the source)."""
    with open(bench.TRAFFIC_RECORD) as f:
        keys = dict(line.split(": ", 1) for line in f.read().splitlines() if ": " in line and not line.startswith("#"))
    assert int(keys["traffic_bytes_per_launch"]) > 0
    assert len(keys["source_md5"].split()[0]) == 12


def test_reference_arm_prints_one_line_of_its_own_sample():
    wl = rime_synth.custom(5, 2, 3, 2, 1, seed_index=90)
    args = argparse.Namespace(gpus=1, steps=2, warmup=1)
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(args, wl, 0, 1) == 0
    lines = [l for l in buf.getvalue().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["ms_per_step"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    # other ranks print nothing
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(args, wl, 1, 2) == 0
    assert buf.getvalue() == ""
