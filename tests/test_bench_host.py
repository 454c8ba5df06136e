"""Host logic of bench.py: the recorded-traffic lookup (kernel source hash and
plan must match the capture) and the parsing of the clock samples taken
during the timed region.  No GPU."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _fake_tree(tmp_path, bench, entry_plan):
    src = tmp_path / "k.cu"
    src.write_text("kernel source v1\n")
    (tmp_path / "profiles").mkdir()
    saved = bench.ROOT
    bench.ROOT = str(tmp_path)
    try:
        h = bench.kernel_hash(["k.cu"])
    finally:
        bench.ROOT = saved
    rec = {"w": {"kernel_hash": h, "dram_bytes_per_launch": 1234}}
    if entry_plan is not None:
        rec["w"]["plan"] = entry_plan
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    return src


def test_traffic_needs_matching_sources(tmp_path, bench, monkeypatch):
    src = _fake_tree(tmp_path, bench, None)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("w", ["k.cu"]) == 1234
    assert bench.recorded_traffic("other", ["k.cu"]) is None
    src.write_text("kernel source v2\n")   # the kernel changed since the capture
    assert bench.recorded_traffic("w", ["k.cu"]) is None


def test_traffic_needs_matching_plan(tmp_path, bench, monkeypatch):
    _fake_tree(tmp_path, bench, {"tile_rows": 128, "sweeps_per_launch": 8})
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("w", ["k.cu"], {"tile_rows": 128, "sweeps_per_launch": 8, "grid": 304}) == 1234
    assert bench.recorded_traffic("w", ["k.cu"], {"tile_rows": 64, "sweeps_per_launch": 8}) is None
    assert bench.recorded_traffic("w", ["k.cu"], None) is None


def test_committed_traffic_records_are_well_formed(bench):
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        recs = json.load(f)
    assert recs
    for name, r in recs.items():
        assert r["dram_bytes_per_launch"] == r["dram_bytes_read"] + r["dram_bytes_write"], name
        assert len(r["kernel_hash"]) == 16
        assert os.path.exists(os.path.join(ROOT, "profiles", r["source"])), name


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_median_and_reasons(bench):
    cs = bench.ClockSampler(0)
    cs.proc = _Done()
    cs.lines = [
        "2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    out = cs.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    cs = bench.ClockSampler(0)
    cs.proc = _Done()
    cs.lines = ["1200, 2070, 700.0, 0x40, Active, Not Active, Not Active, Not Active"]
    assert cs.stop()["reasons"] == ["hw_slowdown"]


def test_clock_sampler_without_nvidia_smi(bench):
    cs = bench.ClockSampler(0)
    out = cs.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]
