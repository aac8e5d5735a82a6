"""bench.py's host-side measurement logic on CPU: the clock sampler's summary (median
SM clock, throttle reasons that reject a run), the gating of the recorded ncu DRAM
bytes and tensor-pipe shares (precision, sample count, kernel-source digest), and
the algorithmic bytes per sample of the field kernels."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(rows):
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.proc = _FakeProc()
    s.rows = rows
    return s


def _row(sm, mx, hw="Not Active", hw_th="Not Active", sw_th="Not Active", pcap="Not Active"):
    return ["0", str(sm), str(mx), "900.0", "0x0", hw, hw_th, sw_th, pcap]


def test_clock_summary_median_and_no_reasons():
    out = _sampler([_row(2070, 2070), _row(2055, 2070), _row(2070, 2070)]).stop()
    assert out["sm_mhz"] == 2070 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == [] and out["samples"] == 3


def test_clock_summary_reports_every_active_reason():
    rows = [_row(1800, 2070, pcap="Active"), _row(1500, 2070, hw_th="Active"), _row(2070, 2070)]
    out = _sampler(rows).stop()
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert out["sm_mhz"] == 1800


def test_clock_summary_without_nvidia_smi():
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.proc = None
    s.rows = []
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_measured_traffic_gating(monkeypatch):
    n = bench.NCU_TRAFFIC["samples"]
    if bench.kernel_sources_digest() != bench.NCU_TRAFFIC["sha256"]:
        pytest.skip("kernel sources changed since the recorded capture")
    full = bench.measured_traffic("field_bwd", "fp16", n)
    assert full == bench.NCU_TRAFFIC["field_bwd"]
    assert bench.measured_traffic("field_bwd", "fp16", int(n * 1.01)) == pytest.approx(full * 1.01, rel=1e-6)
    assert bench.measured_traffic("field_bwd", "fp16", int(n * 1.03)) is None     # another workload
    assert bench.measured_traffic("field_bwd", "bf16", n) is None                 # another precision
    assert bench.measured_traffic("adam", "fp16", n) is None                      # not captured
    assert bench.measured_tensor_pipe("fp16")["field_bwd"] == bench.NCU_TRAFFIC["tensor_pipe"]["field_bwd"]
    monkeypatch.setitem(bench.NCU_TRAFFIC, "sha256", "0" * 64)                    # sources edited
    assert bench.measured_traffic("field_bwd", "fp16", n) is None
    assert bench.measured_tensor_pipe("fp16") is None


@pytest.mark.parametrize("prec,enc", [("fp16", 64), ("bf16", 64), ("fp32", 128)])
def test_algorithmic_bytes_per_sample(prec, enc):
    cfg = synth.config_c2(prec)
    b = bench.algorithmic_bytes(cfg, 1000, 10)
    table = 8 * 16 * 2 * 4                       # 8 corners x 16 levels x 2 FP32 features
    assert b["field_fwd"] == 1000 * (table + 8 + enc + 16)
    assert b["field_bwd"] == 1000 * (table + 8 + enc + 32)
    assert b["adam"] == 320
    if prec == "fp16":
        assert b["field_fwd"] // 1000 == 1112 and b["field_bwd"] // 1000 == 1128


def test_replica_throughput_counts_every_replica():
    assert bench.replica_throughput(262144, 4, 0.5) == 262144 * 4 / 0.5
    assert bench.max_over_ranks(None, 3.5) == 3.5
