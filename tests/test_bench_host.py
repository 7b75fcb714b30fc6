"""Host-side pieces of bench.py that need no GPU: the kernel name reported
for each step-a variant (it must match ncu's name for the same kernel) and the
rule that a recorded DRAM-traffic figure is reported only for the kernel
sources it was measured on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("var,name", [
    (0, "cg_step_a_kernel<float, 12, 0>"),
    (4, "cg_step_a_kernel<float, 12, 4>"),
    (5, "cg_step_a_staged_kernel<float, 12, 2, 0, 0>"),
    (6, "cg_step_a_staged_kernel<float, 12, 4, 0, 0>"),
    (7, "cg_step_a_staged_kernel<float, 12, 2, 1, 0>"),
    (8, "cg_step_a_staged_kernel<float, 12, 3, 0, 1>"),
])
def test_kernel_name_per_variant(var, name):
    assert bench.step_a_kernel_name({"step_a_variant": var, "k_bucket": 12}) == name


def test_recorded_traffic_needs_matching_kernel_and_sources(tmp_path, monkeypatch):
    note = tmp_path / "note.md"
    h = bench.kernel_source_hash()
    note.write_text("text\ntraffic_per_launch: kernel=K<float, 12, 4, 0, 0>; bytes=123; source_sha256=%s\n" % h)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path.parent))
    monkeypatch.setattr(bench, "TRAFFIC_NOTE", os.path.join(tmp_path.name, "note.md"))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.recorded_traffic("K<float, 12, 4, 0, 0>") == 123
    assert bench.recorded_traffic("K<float, 12, 2, 0, 0>") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.recorded_traffic("K<float, 12, 4, 0, 0>") is None


def test_committed_note_parses():
    """The committed ncu summary carries a well-formed traffic line."""
    path = os.path.join(ROOT, bench.TRAFFIC_NOTE)
    lines = [l for l in open(path) if l.startswith("traffic_per_launch:")]
    assert len(lines) == 1
    kv = dict(x.strip().split("=", 1) for x in lines[0].split(":", 1)[1].split(";"))
    assert set(kv) == {"kernel", "bytes", "source_sha256"} and int(kv["bytes"]) > 0
