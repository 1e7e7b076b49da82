"""Host-side bookkeeping of bench.py (no GPU): the committed ncu figures
that go into the roofline line are used only while the kernel sources they
were taken on are unchanged, each summary only for its own precision, and
DRAM traffic is scaled to the launch's particle count."""
import os
import shutil

import bench


def test_kernel_hash_covers_the_kernel_sources(tmp_path, monkeypatch):
    h0 = bench.kernel_hash()
    csrc = os.path.join(bench.ROOT, "paper_2512_02175_gb300", "csrc")
    root = tmp_path / "r"
    shutil.copytree(csrc, root / "paper_2512_02175_gb300" / "csrc")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.kernel_hash() == h0
    for f in ("mg_em_step.cuh", "mg_types.h", "mg_log_table.h"):
        p = root / "paper_2512_02175_gb300" / "csrc" / f
        text = p.read_text()
        p.write_text(text + "\n// changed\n")
        assert bench.kernel_hash() != h0, f
        p.write_text(text)
    assert bench.kernel_hash() == h0


def test_profile_figures():
    """The committed summaries' figures, while they match the kernel
    sources (after a kernel change the benchmark reports traffic null until
    the kernel is profiled again)."""
    import pytest
    h = bench.kernel_hash()
    mixed = bench._profile(h)
    fp64 = bench._profile(h, "em_step_star16_fp64.md")
    if not (mixed and fp64):
        pytest.skip("the committed ncu summaries were taken on other kernel sources")
    assert 0.0 < float(mixed["issue-active-pct"]) <= 100.0
    assert 0.0 < float(fp64["fp64-pipe-active-pct"]) <= 100.0
    assert "fp64-pipe-active-pct" not in mixed


def test_profile_ignored_when_stale():
    assert bench._profile("0" * 64) == {}
    assert bench._profile("0" * 64, "em_step_star16_fp64.md") == {}


def test_traffic_scales_with_particles():
    prof = {"dram-bytes-per-launch-full-size": str(1 << 30)}
    assert bench._traffic(prof, bench.PROFILE_N) == 1 << 30
    assert bench._traffic(prof, bench.PROFILE_N // 4) == 1 << 28
    assert bench._traffic({}, 123) is None
