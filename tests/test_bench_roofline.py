"""Host logic of bench.py's roofline report (no GPU): the dominant stage, the
achieved rate from algorithmic bytes and time, the traffic scaling, and the
operator byte count against an independent count over the chains."""

import pytest

pytest.importorskip("torch")
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6790.3}


def test_operator_bytes_match_chain_count():
    ns, L, B = 64, 128, 40
    p = 2 * ns
    P2 = p // 2 + 1
    rows = sum(bench.chain_len(m, c, L) for m in range(L + 1) for c in (0, 1))
    nalm = (L + 1) * (L + 2) // 2
    assert rows == nalm
    kind, amount = bench.stage_work(ns, L, B)["fused_fsht"]
    # two column tiles of 32 maps read M twice; b and alm once per map
    expect = 2 * rows * P2 * 4 + B * (L + 1) * 2 * P2 * 8 + B * nalm * 8
    assert kind == "hbm" and amount == expect


def test_dominant_stage_and_rates():
    work = bench.stage_work(1024, 2048, 32)
    per_launch = {"ring_fft": 2.51, "poles": 0.008, "spread": 1.05, "lat_fft": 1.66, "fused_fsht": 2.43,
                  "unused": 0.002}
    roof, stages = bench.roofline_report(work, per_launch, PEAKS)
    assert roof["kernel"] == "ring_fft"
    amount = work["ring_fft"][1]
    assert roof["achieved"] == pytest.approx(amount / 2.51e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 6790.3)
    # traffic: the ring stage's DRAM bytes per algorithmic byte (ncu at Nside 512), scaled
    assert roof["traffic"] == pytest.approx(amount * bench.TRAFFIC_OVER_ALGORITHMIC["ring_fft"])
    assert "unused" not in stages and set(stages) == {"ring_fft", "poles", "spread", "lat_fft", "fused_fsht"}
    op = stages["fused_fsht"]
    assert op["frac"] == pytest.approx(work["fused_fsht"][1] / 2.43e-3 / 1e9 / 6790.3)
    assert 0.5 < op["frac"] < 0.7               # 10.2 GB in 2.43 ms


def test_traffic_scaled_for_captured_kernel():
    work = bench.stage_work(1024, 2048, 32)
    per_launch = {"ring_fft": 2.0, "spread": 1.0, "lat_fft": 1.5, "fused_fsht": 2.4}
    roof, _ = bench.roofline_report(work, per_launch, PEAKS)
    assert roof["kernel"] == "fused_fsht"
    ratio = bench.TRAFFIC_OVER_ALGORITHMIC["fused_fsht"]
    assert roof["traffic"] == pytest.approx(work["fused_fsht"][1] * ratio)
    assert 1.0 <= ratio < 1.2                   # padding only: no re-reads
    # the operator stage is compute-bound under the survey's accounting: the flops of D and the sweeps
    assert roof["bound"] == "tensor"
    flops = work["lat_solve"][1] + work["rot_sweep"][1]
    assert roof["achieved"] == pytest.approx(flops / 2.4e-3 / 1e12)
    assert roof["operator_stream"]["bytes"] == work["fused_fsht"][1]


def test_fallback_peak_without_measurements():
    work = bench.stage_work(64, 128, 8)
    roof, _ = bench.roofline_report(work, {"spread": 1.0, "lat_fft": 0.5}, {})
    assert roof["peak_source"] == "fallback" and roof["peak"] == 6800.0


def test_cpu_cost_model_separates_fixed_and_per_order_time():
    """The oracle's time for n orders is fixed + n * per_order; two sample sizes
    recover both, and the full map is fixed + 2049 * per_order (not the small
    sample's time scaled by 2049 / n, which counts the fixed part 2049 / n times)."""
    fixed, per = bench.fit_cost_model(2, 7.0 + 2 * 0.5, 16, 7.0 + 16 * 0.5)
    assert abs(fixed - 7.0) < 1e-12 and abs(per - 0.5) < 1e-12
    assert abs(bench.full_map_seconds(fixed, per) - (7.0 + 2049 * 0.5)) < 1e-9
    assert abs(bench.cpu_gpix(100.0) - 12 * 1024 * 1024 / 100.0 / 1e9) < 1e-18
