"""bench.py's use of the committed ncu record: the DRAM traffic and the
executed instruction count of a step are reported only while the kernel
sources match the digest they were captured on (and the schedule matches),
scaled by the site count, and documentation edits do not invalidate them
(CPU only)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_committed_record_matches_the_current_kernel_sources():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)["d3q19-256"]
    assert rec["sources_sha256"] == bench.sources_digest()
    cap = bench.recorded_capture("d3q19-256", 256 ** 3, rec["schedule"])
    scale = 256 ** 3 / rec["sites"]
    assert cap["traffic"] == rec["dram_bytes_per_step"] * scale
    assert cap["inst"] == rec["warp_instructions_per_step"] * scale
    assert bench.recorded_capture("d3q19-256", 256 ** 3, "some other schedule") is None


def test_record_is_ignored_for_other_sources(tmp_path, monkeypatch):
    src = os.path.join(ROOT, "paper_1410_5584_gb300", "csrc")
    copy = tmp_path / "paper_1410_5584_gb300" / "csrc"
    copy.mkdir(parents=True)
    for name in os.listdir(src):
        if name.endswith((".cu", ".cuh", ".h")):
            (copy / name).write_text(open(os.path.join(src, name), encoding="utf-8").read())
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(open(os.path.join(ROOT, "profiles", "traffic.json")).read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_capture("d3q19-256", 8) is not None
    # a comment does not change the digest; code does
    k = copy / "flbm_kernels.cuh"
    k.write_text(k.read_text() + "\n// a note\n")
    assert bench.recorded_capture("d3q19-256", 8) is not None
    k.write_text(k.read_text() + "\nstatic const int kChanged = 1;\n")
    assert bench.recorded_capture("d3q19-256", 8) is None
    assert bench.recorded_capture("d2q9-512", 8) is None
