"""The bench's roofline inputs from the committed ncu record: DRAM bytes and
ALU-pipe instructions per launch are reported only while every source of
the kernel still has the recorded hash, and the ALU fraction is instructions over time
against 152 SMs x 2 warp-instructions per clock x 2070 MHz."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _record_at(tmp_path, monkeypatch, source_text=None):
    """A copy of the committed record under tmp_path whose stage_b source is
    a file there (its hash recorded, or made stale by `source_text`)."""
    import hashlib
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    src = tmp_path / "k.cu"
    src.write_text("// a kernel\n")
    rec["stage_b"]["sources"] = {str(src): hashlib.sha256(src.read_bytes()).hexdigest()}
    if source_text is not None:
        src.write_text(source_text)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return rec


def test_record_matches_the_sources():
    # the committed record describes the committed kernels (else the bench
    # reports no traffic: a capture of the changed kernel is due)
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        rec = json.load(fh)
    for stage in ("stage_a", "stage_b"):
        if bench.measured_counters(stage) is None:
            pytest.skip(f"{stage}: kernel source changed since the ncu capture")
        assert bench.measured_traffic(stage) == rec[stage]["dram_read_bytes"] + rec[stage]["dram_write_bytes"]


def test_alu_roofline_arithmetic(tmp_path, monkeypatch):
    rec = _record_at(tmp_path, monkeypatch)
    alu = bench.alu_roofline("stage_b", 0.1)
    want = rec["stage_b"]["alu_pipe_warp_insts"] / 1e-4 / 1e9
    assert abs(alu["achieved"] - round(want, 1)) < 0.11
    assert alu["peak"] == round(152 * 2 * 2.070, 1)
    assert abs(alu["frac"] - want / (152 * 2 * 2.070)) < 1e-4
    assert bench.alu_roofline("stage_b", 0) is None


def test_changed_source_hides_the_record(tmp_path, monkeypatch):
    _record_at(tmp_path, monkeypatch, source_text="// a changed kernel\n")
    assert bench.measured_counters("stage_b") is None
    assert bench.measured_traffic("stage_b") is None
    assert bench.alu_roofline("stage_b", 0.1) is None


def test_any_changed_source_hides_the_record(tmp_path, monkeypatch):
    # a kernel built from two files (stage A: its kernel and the float unit
    # it inlines) is reported only while both still have their hashes
    import hashlib
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    a, b = tmp_path / "a.cu", tmp_path / "b.cuh"
    a.write_text("// kernel\n")
    b.write_text("// its header\n")
    rec["stage_a"]["sources"] = {str(f): hashlib.sha256(f.read_bytes()).hexdigest() for f in (a, b)}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("stage_a") == rec["stage_a"]["dram_read_bytes"] + rec["stage_a"]["dram_write_bytes"]
    b.write_text("// its header, changed\n")
    assert bench.measured_traffic("stage_a") is None
