"""Host-side logic of bench.py (no GPU): the argument defaults and the lookup
of the committed ncu traffic figures, which must be dropped once the kernel
sources differ from the ones the counters were taken on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_defaults(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert (a.gpus, a.impl, a.precision, a.separate) == (1, "ours", "fp64", False)
    assert a.warmup >= 3 and a.steps >= 1


def test_every_headline_form_has_a_profile_summary():
    for form, path in bench.PROFILES.items():
        assert os.path.exists(path), form
        text = open(path).read()
        assert "kernel_sources_sha:" in text and "dram_bytes_per_step:" in text, form
        assert "--clock-control none" in text, form


@pytest.mark.parametrize("matching", [True, False])
def test_profile_traffic_only_for_the_current_sources(tmp_path, monkeypatch, matching):
    sha = bench.kernel_sources_sha()
    f = tmp_path / "k.txt"
    f.write_text("Kernel: k\nkernel_sources_sha: %s\ndram_bytes_per_step: 3.5e8\n" % (sha if matching else "0" * 16))
    monkeypatch.setitem(bench.PROFILES, "fp64_fused", str(f))
    got = bench.read_profile_traffic("fp64_fused")
    assert got == (3.5e8 if matching else None)


def test_missing_profile_gives_no_traffic(monkeypatch, tmp_path):
    monkeypatch.setitem(bench.PROFILES, "mixed", str(tmp_path / "absent.txt"))
    assert bench.read_profile_traffic("mixed") is None
