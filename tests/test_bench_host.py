"""Host-side arithmetic of the benchmark line, on the CPU: the algorithmic FLOP
count per point, the per-pass rooflines (achieved = FLOPs / time, fraction of the
stated peak, the longest pass on top), the peak fallback, and the library's
kernel count per verify call."""
import json

import pytest

import bench


def test_flops_per_point_counts_dense_layers_and_table_adds():
    # 784-512-512-10, s = 6: 2 (512*512 + 512*10) + 6*512 = 537,600
    assert bench.screen_flops_per_point([784, 512, 512, 10], 6) == 537_600
    # a net without dense layers after layer 1 does s * H_1 table adds only
    assert bench.screen_flops_per_point([25, 10], 5) == 50
    # 25-10-5, s = 5: 2 * 10 * 5 + 5 * 10
    assert bench.screen_flops_per_point([25, 10, 5], 5) == 150


def _sums(ms_screen, ms_pass, n_recheck):
    return [{"ms_screen": ms_screen, "ms_pass": list(ms_pass), "n_recheck": list(n_recheck)}]


def test_pass_rooflines_bf16():
    dims, s, n = [784, 512, 512, 10], 6, 11_390_625
    pk = {"bf16_tflops": 2000.0, "sm_max_mhz": 2000.0}
    sums = _sums(20.0, [10.0, 25.0, 5.0, 0.5], [3_000_000, 1_000_000, 40_000, 50])
    traffic = {"screen (first pass over every point)": 1000, "FP32 pass": 7}
    r = bench.pass_rooflines("bf16", dims, s, n, sums, pk, "measured", traffic)
    by = {p["kernel"]: p for p in r["passes"]}
    fpp = 537_600
    alu = 152 * 128 * 2 * 2000.0e6 / 1e12  # 77.824 TFLOP/s
    exp = {
        "screen (first pass over every point)": (fpp * n, 20.0, 2000.0),
        "split tensor pass": (fpp * 3_000_000, 10.0, 2000.0),
        "FP32 pass": (fpp * 1_000_000, 25.0, alu),
        "double-float pass": (fpp * 40_000, 5.0, alu * 2 / 11),
        "FP64 pass": (fpp * 50, 0.5, 1.25),
    }
    for name, (flops, ms, peak) in exp.items():
        p = by[name]
        assert p["flops_per_launch"] == flops
        assert p["achieved"] == pytest.approx(flops / (ms / 1e3) / 1e12)
        assert p["peak"] == pytest.approx(peak)
        assert p["frac"] == pytest.approx(p["achieved"] / peak)
    # the split pass: one evaluation per point is the method's work; its three
    # products per layer are reported as hardware work beside it
    assert by["split tensor pass"]["hardware_flops_per_launch"] == 3 * fpp * 3_000_000
    assert "hardware_flops_per_launch" not in by["FP32 pass"]
    assert by["screen (first pass over every point)"]["traffic"] == 1000
    assert by["FP32 pass"]["traffic"] == 7 and by["split tensor pass"]["traffic"] is None
    # the top-level fields are those of the longest pass (the FP32 pass here)
    assert r["kernel"] == "FP32 pass" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["frac"] == by["FP32 pass"]["frac"] and r["traffic"] == 7


def test_pass_rooflines_skips_passes_that_did_not_run_and_scales_fp8():
    pk = {"bf16_tflops": 1000.0, "sm_max_mhz": 2070.0}
    sums = _sums(30.0, [0.0, 2.0, 0.0, 0.0], [0, 100, 0, 0])
    r = bench.pass_rooflines("fp8", [784, 1024, 1024, 1024, 10], 5, 1000, sums, pk, "measured")
    names = [p["kernel"] for p in r["passes"]]
    assert names == ["screen (first pass over every point)", "FP32 pass"]
    assert r["kernel"] == "screen (first pass over every point)"
    assert r["peak"] == pytest.approx(2000.0)  # E4M3: twice the BF16 figure
    assert r["traffic"] is None


def test_plain_fp32_path_puts_the_screen_on_the_alu_roof():
    pk = {"bf16_tflops": 1000.0, "sm_max_mhz": 2070.0}
    r = bench.pass_rooflines("fp32", [784, 512, 512, 10], 6, 1000, _sums(5.0, [0, 0, 1.0, 0.1], [0, 0, 10, 1]),
                             pk, "measured")
    top = r["passes"][0]
    assert top["bound"] == "alu" and top["peak"] == pytest.approx(152 * 128 * 2 * 2070.0e6 / 1e12)


def test_peaks_fallback_and_measured(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    pk, kind = bench.peaks()
    assert kind == "fallback" and pk["hbm_gbs"] == 6800.0 and pk["bf16_tflops"] == 1900.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 1.0, "bf16_tflops": 2.0}))
    pk, kind = bench.peaks()
    assert kind == "measured" and pk == {"hbm_gbs": 1.0, "bf16_tflops": 2.0}


def test_launches_per_verify_call():
    # BF16 chain of a 3-layer net: prologue (init, 3 base layers, tables, finish),
    # column classes, screen, split, FP32, double-float, FP64, time stamps
    assert bench.launches_per_step("bf16", 3) == 13
    assert bench.launches_per_step("bf16", 3, batch=True) == 12
    assert bench.launches_per_step("fp32", 3) == 10
    assert bench.launches_per_step("fp64", 3) == 8
    # E4M3: per chunk of 2^20 points layer 1, GEMM + stats per hidden layer >= 2,
    # output layer and three recheck passes
    assert bench.launches_per_step("fp8", 4, n_points=3 << 20) == 7 + 3 * (1 + 4 + 1 + 3) + 2


def test_profiled_traffic_is_keyed_by_the_bench_configuration():
    for key, per_pass in bench.PROFILED_TRAFFIC.items():
        workload, precision, coverage, s, k = key
        assert isinstance(workload, str) and precision in ("bf16", "fp16", "fp8", "fp32")
        assert isinstance(coverage, bool) and s >= 1 and k >= 1
        assert set(per_pass) <= {"screen (first pass over every point)", "split tensor pass", "FP32 pass",
                                 "double-float pass", "FP64 pass"}
        assert all(isinstance(v, int) and v > 0 for v in per_pass.values())


def test_reference_arm_times_each_step_on_its_own_sample(monkeypatch):
    """--impl reference: K timed steps, each one contiguous sample of the query;
    ms_per_step is those steps' mean time and the rate counts only their points."""
    import synth
    w = synth.workload("mlp25_sigmoid_s5k8", s=3, k=4)
    rate, ms_step, m, cores, sample = bench.oracle_steps(w["net"], w["query"], steps=3, warmup=1,
                                                        seconds_total=0.3)
    n = 9 ** 3
    assert 1 <= m <= n and cores >= 1
    assert rate == pytest.approx(m / (ms_step / 1e3), rel=1e-9)
    assert sample.startswith(f"3 steps of {m} contiguous points")


def test_passes_without_their_own_time_are_left_out():
    """The wide-layer path rechecks each chunk's points inside the first pass's
    timed region: those passes carry no separate time (a few microseconds of
    event markers) and get no roofline of their own; they are named instead."""
    dims, s, n = [784, 1024, 1024, 1024, 10], 5, 28_629_151
    pk = {"bf16_tflops": 2000.0, "sm_max_mhz": 2000.0}
    sums = _sums(5000.0, [0.002, 0.002, 0.002, 0.006], [0, 27_989_462, 619_518, 1316])
    r = bench.pass_rooflines("bf16", dims, s, n, sums, pk, "measured")
    names = [p["kernel"] for p in r["passes"]]
    assert "FP32 pass" not in names and "double-float pass" not in names and "FP64 pass" not in names
    assert r["passes_timed_in_screen"] == ["FP32 pass", "double-float pass", "FP64 pass"]
    assert r["kernel"] == "screen (first pass over every point)"
    assert r["frac"] < 1.0
