"""The benchmark's DRAM-traffic figures come from the committed ncu summaries
only while the kernel sources they were taken on are unchanged (CPU)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def read_kv(path):
    kv = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                key, val = line.split(":", 1)
                kv[key.strip()] = val.strip()
    return kv


@pytest.mark.parametrize("key", sorted(bench.PROFILES))
def test_profiles_parse_and_scale(key):
    kv = read_kv(bench.PROFILES[key])
    per_capture = float(kv["dram_bytes_per_launch_capture"])
    capture_n = float(kv["capture_n"])
    full = float(kv["dram_bytes_per_launch_full"])
    # traffic grows with n: the 1e6-point figure is the capture scaled
    assert full == pytest.approx(per_capture * 1e6 / capture_n, rel=1e-6)
    assert len(kv["source_hash"]) == 16


def test_traffic_only_on_the_captured_sources(monkeypatch):
    h = bench.kernel_source_hash()
    fresh = {key: read_kv(path)["source_hash"] == h for key, path in bench.PROFILES.items()}
    for key, ok in fresh.items():
        got = bench.profile_traffic(*key)
        assert (got is not None) == ok
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    for key in bench.PROFILES:
        assert bench.profile_traffic(*key) is None


def test_hash_covers_the_profiled_kernel_sources():
    csrc = os.path.join(ROOT, "paper_2201_00701_gb300", "csrc")
    for name in bench.KERNEL_SOURCES:
        assert os.path.isfile(os.path.join(csrc, name)), name
    assert bench.kernel_source_hash() == bench.kernel_source_hash()
