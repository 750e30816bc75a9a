"""bench.py's host-side pieces that need no GPU: the throttle-reason decoding
of the clock record (a run that saw hw_slowdown, hw_thermal_slowdown or
sw_thermal_slowdown must show it; sw_power_cap is kept and noted) and the
traffic lookup keyed by the sweep kernel's source hash."""
import json

import pytest

import bench


class _Out:
    def __init__(self, stdout):
        self.stdout = stdout


def _sampler(monkeypatch, lines):
    it = iter(lines)
    monkeypatch.setattr(bench.subprocess, "run", lambda *a, **k: _Out(next(it)))
    c = bench.ClockSampler(0)
    c._nvml = None             # the nvidia-smi path
    return c


def test_smi_reasons_decode_in_query_order(monkeypatch):
    # query columns: clocks.sm, clocks.max.sm, hw_slowdown, hw_thermal_slowdown,
    # sw_thermal_slowdown, sw_power_cap
    c = _sampler(monkeypatch, ["2070, 2070, Not Active, Not Active, Not Active, Active",
                               "1980, 2070, Not Active, Not Active, Not Active, Not Active",
                               "2070, 2070, Not Active, Not Active, Not Active, Not Active"])
    for _ in range(3):
        c._sample_smi()
    s = c.summary()
    assert s["reasons"] == ["sw_power_cap"] and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["samples"] == 3 and s["source"] == "nvidia-smi"


@pytest.mark.parametrize("col,name", [(2, "hw_slowdown"), (3, "hw_thermal_slowdown"),
                                      (4, "sw_thermal_slowdown")])
def test_smi_rejecting_reasons_are_reported(monkeypatch, col, name):
    f = ["1500", "2070", "Not Active", "Not Active", "Not Active", "Not Active"]
    f[col] = "Active"
    c = _sampler(monkeypatch, [", ".join(f)])
    c._sample_smi()
    assert c.summary()["reasons"] == [name]


def test_smi_unparseable_line_is_skipped(monkeypatch):
    c = _sampler(monkeypatch, ["[N/A], [N/A], [N/A], [N/A], [N/A], [N/A]"])
    c._sample_smi()
    s = c.summary()
    assert s["samples"] == 0 and s["sm_mhz"] is None and s["reasons"] == []


def test_traffic_lookup_needs_the_current_kernel_source(tmp_path, monkeypatch):
    path = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(path))
    path.write_text(json.dumps({"road2048": {"dram_bytes_per_launch": 123,
                                             "source_hash": bench.sweep_source_hash()}}))
    assert bench.profiled_traffic("road2048") == 123
    assert bench.profiled_traffic("rmat22") is None
    path.write_text(json.dumps({"road2048": {"dram_bytes_per_launch": 123, "source_hash": "0" * 16}}))
    assert bench.profiled_traffic("road2048") is None
