"""bench.py's use of the committed ncu figures (profiles/traffic.json), on CPU: they count only
while the kernel's sources hash matches the one they were taken with, they scale with the
element count, and the issue view divides the scaled warp instructions by the launch time
against four issue slots per SM per clock."""
import json
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import bench  # noqa: E402


def _fake_profiles(tmp_path, monkeypatch, entries, current_hash="h-current"):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(entries))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "sources_hash", lambda kernel, read=None: current_hash)


def test_counters_scale_with_the_element_count(tmp_path, monkeypatch):
    _fake_profiles(tmp_path, monkeypatch, {
        "mass_f64_soa": {"bytes_per_launch": 4.0e9, "warp_inst_per_launch": 2.0e9,
                         "sources_hash": "h-current"}})
    assert bench._profile_traffic("mass_f64_soa", bench.PROFILE_N) == pytest.approx(4.0e9)
    assert bench._profile_traffic("mass_f64_soa", bench.PROFILE_N // 4) == pytest.approx(1.0e9)
    r = bench.issue_roofline("mass_f64_soa", 2.0, 2000.0, 152, bench.PROFILE_N // 2)
    assert r["warp_inst_per_launch"] == pytest.approx(1.0e9)
    assert r["achieved"] == pytest.approx(1.0e9 / 2.0e-3)
    assert r["peak"] == pytest.approx(4 * 152 * 2000.0e6)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # without a sampled SM clock there is no issue peak to compare against
    assert bench.issue_roofline("mass_f64_soa", 2.0, None, 152, bench.PROFILE_N) is None


def test_counters_of_other_sources_are_not_used(tmp_path, monkeypatch):
    _fake_profiles(tmp_path, monkeypatch, {
        "mass_f64_soa": {"bytes_per_launch": 4.0e9, "warp_inst_per_launch": 2.0e9,
                         "sources_hash": "h-old"}})
    assert bench._profile_traffic("mass_f64_soa", bench.PROFILE_N) is None
    assert bench.issue_roofline("mass_f64_soa", 2.0, 2000.0, 152, bench.PROFILE_N) is None
    # a kernel bench.py does not time gives nothing either
    assert bench._profile_traffic("no_such_kernel", bench.PROFILE_N) is None


def test_missing_or_broken_file_gives_no_counters(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._profile_traffic("mass_f64_soa", bench.PROFILE_N) is None
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text("{not json")
    assert bench._profile_traffic("mass_f64_soa", bench.PROFILE_N) is None


def test_sources_hash_follows_every_source_file():
    """The hash changes with the content of each file the kernel is built from, and only with
    those: the committed figures go stale exactly when a kernel source changes."""
    files = bench.KERNEL_SOURCES["mass_f64_soa"]
    base = bench.sources_hash("mass_f64_soa", read=lambda rel: b"x")
    for f in files:
        changed = bench.sources_hash("mass_f64_soa", read=lambda rel: b"y" if rel == f else b"x")
        assert changed != base, f
    # the boost is built from other files: its hash does not move with the mass-only sources
    boost_files = set(bench.KERNEL_SOURCES["boost_f64_soa"])
    only_mass = [f for f in files if f not in boost_files]
    assert only_mass
    b0 = bench.sources_hash("boost_f64_soa", read=lambda rel: b"x")
    b1 = bench.sources_hash("boost_f64_soa",
                            read=lambda rel: b"y" if rel in only_mass else b"x")
    assert b0 == b1


def test_every_kernel_source_exists():
    csrc = os.path.join(os.path.dirname(HERE), "paper_2312_02756_gb300", "csrc")
    for kernel, files in bench.KERNEL_SOURCES.items():
        for f in files:
            assert os.path.isfile(os.path.join(csrc, f)), (kernel, f)
