"""Host-side logic of bench.py that needs no GPU: the clock-sample summary
(median SM clock, throttle reasons, power) and the hash-gated DRAM traffic
record that feeds `roofline.traffic`."""
import hashlib
import json
import os

import bench
from paper_1010_0012_gb300 import workload as wl


def _line(sm, mx, pw, active="Not Active", hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, {pw}, {active}, {hw}, {hwt}, {swt}, {cap}"


def test_clock_summary_median_reasons_and_power():
    c = bench.ClockSampler(0)
    c.lines = [_line(2070, 2070, 600.5), _line(1980, 2070, 900.0, cap="Active"),
               _line(2070, 2070, 700.0), "garbage", _line("[N/A]", 2070, 1.0)]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 3
    assert s["power_w"] == 700.0


def test_clock_summary_flags_every_slowdown_reason():
    c = bench.ClockSampler(0)
    c.lines = [_line(1500, 2070, 1000, hw="Active"), _line(1500, 2070, 1000, hwt="Active"),
               _line(1500, 2070, 1000, swt="Active")]
    assert c.summary()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    s = bench.ClockSampler(0).summary()
    assert s["samples"] == 0 and s["sm_mhz"] is None and s["reasons"] == []


def test_traffic_record_is_reported_only_for_the_current_sources(tmp_path, monkeypatch):
    cfg = wl.CONFIGS["grid1280x720_m128"]
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    rec = {"band_sum_kernel<16,2,4>": {"source_files": ["k.cu"], "dram_bytes_full_launch": 123,
                                        "source_sha256": hashlib.sha256(b"kernel v1").hexdigest()}}
    os.makedirs(tmp_path / "profiles")
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("band_sum_kernel<16,2,4>", cfg) == 123
    assert bench.recorded_traffic("band_sum_kernel<32,1,4>", cfg) is None       # no record for this kernel
    src.write_text("kernel v2")                                                  # source changed since the capture
    assert bench.recorded_traffic("band_sum_kernel<16,2,4>", cfg) is None


def test_algorithmic_bytes_and_units_of_the_benchmark_workload():
    cfg = wl.CONFIGS["grid1280x720_m128"]
    De = wl.directed_edges(cfg.W, cfg.H)
    assert De == 2 * (720 * 1279 + 1280 * 719)
    assert bench.workload_units(cfg) == De * 128
    assert bench.algorithmic_bytes(cfg) == (1280 * 720 * 128 + 2 * De * 128) * 4 == 4242636800


def test_gradient_floor_counts_each_launch_of_the_checkpointed_schedule():
    """256x256, M = 64, K = 30, checkpoint 5: 30 recorded forward launches
    and 20 recomputed ones (segments 0..4 recompute 4 states each; the last
    segment's states are kept) at (W H M + 2 De M) * 4 bytes, 30 adjoint
    launches at 15 words per node-label, one copy of a 4-plane state."""
    import bench
    from paper_1010_0012_gb300 import workload as wl
    cfg = wl.CONFIGS["grid256_m64_grad"]
    total, parts = bench.gradient_floor_bytes(cfg, 5)
    De = 2 * (256 * 255 + 256 * 255)
    fwd = (256 * 256 * 64 + 2 * De * 64) * 4
    assert fwd == 150_470_656
    assert parts["forward"] == 30 * fwd and parts["recompute"] == 20 * fwd
    assert parts["adjoint"] == 30 * 256 * 256 * 64 * 60
    assert parts["checkpoints"] == 2 * 4 * 256 * 256 * 64 * 4
    assert total == sum(parts.values())


def test_update_bytes_of_the_dense_forms():
    import bench
    assert bench.UPDATE_BYTES["band_mM"] == 9.0
    assert bench.UPDATE_BYTES["dense_bf16_tcgen05_fused"] == 9.0
    assert bench.UPDATE_BYTES["dense_bf16_tcgen05"] == 13.0
