"""Host-side bookkeeping of bench.py: algorithmic bytes, kernel naming and the
hash-gated profile traffic (no GPU needed)."""

import os

import pytest

import bench


def test_algorithmic_bytes_per_instance():
    # detection: H and Y read; x_hat, mu, rho, 6 LLRs per user and the status written
    assert bench.detect_bytes_per_instance(128, 16, 14, 6) == \
        (128 * 16 + 14 * 128) * 8 + 14 * 16 * (8 + 4 + 4 + 6 * 4) + 4 == 39684
    # precoding: H and T read; q, ||q|| and the status written
    assert bench.precode_bytes_per_instance(128, 16, 14) == \
        (128 * 16 + 14 * 16) * 8 + 14 * 128 * 8 + 14 * 4 + 4 == 32572


@pytest.mark.parametrize("precision,U,name", [
    ("fp16x3", 16, "detect_warp_kernel<16, FP16, true>"),
    ("bf16", 8, "detect_warp_kernel<8, BF16, false>"),
    ("bf16x3", 32, "detect_warp_kernel<32, BF16, true>"),
    ("fp32", 16, "detect_kernel<16>")])
def test_detect_kernel_name(precision, U, name):
    assert bench.detect_kernel_name(precision, U) == name


def test_profile_traffic_is_used_only_with_matching_sources(tmp_path, monkeypatch):
    current = bench.kernel_source_hash()   # of the real sources
    (tmp_path / "profiles").mkdir()
    good = tmp_path / "profiles" / "good.md"
    good.write_text(f"kernel_source_hash: {current}\ndram_bytes_per_full_launch: 1.25e9\n")
    stale = tmp_path / "profiles" / "stale.md"
    stale.write_text("kernel_source_hash: 0000000000000000\ndram_bytes_per_full_launch: 1e9\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))   # only the profile lookup moves
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: current)
    assert bench.profiled_traffic("good") == pytest.approx(1.25e9)
    assert bench.profiled_traffic("stale") is None
    assert bench.profiled_traffic("missing") is None


def test_kernel_sources_exist():
    csrc = os.path.join(bench.ROOT, "paper_1404_0424_gb300", "csrc")
    for fn in bench.KERNEL_SOURCES:
        assert os.path.exists(os.path.join(csrc, fn)), fn


def test_every_precision_has_its_dtype_label():
    # the bench line's dtype names the arithmetic of the precision that ran
    assert set(bench.DTYPES) == set(bench.PRECISIONS)
    assert bench.DTYPES["fp32"] == "f32"
    assert bench.DTYPES["fp16x3"].startswith("f16x3")
