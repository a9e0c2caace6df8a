"""Host logic of bench.py's roofline (no GPU): which bound the objective
kernel is reported against, and the arithmetic of each."""
import pytest

import bench


def test_alu_peak_from_unit_counts():
    # 152 SMs x 128 FP32 lanes x 2.07 GHz x 2 flops
    assert bench.ALU_PEAK_TFLOPS == pytest.approx(80.547, rel=1e-4)


def test_split_tf32_form_at_small_k_is_hbm_bound():
    # the fp32 workload's split-TF32 launch as measured: 0.2415 ms for 10^7 x 16
    e = bench.roofline_entry("tcs_objective_kernel", "split_tf32", 10_000_000, 16, 25.0, 0.24152,
                             6785.9, "measured", 648553216.0)
    assert e["bound"] == "hbm" and e["unit"] == "GB/s"
    assert e["achieved"] == pytest.approx(640e6 / 0.24152e-3 / 1e9, rel=1e-12)
    assert e["frac"] == pytest.approx(0.3905, abs=1e-4)
    assert e["traffic"] == 648553216.0 and e["algorithmic_bytes_per_launch"] == 640e6


def test_cuda_core_form_at_large_k_is_alu_bound():
    # the large workload's CUDA-core launch: 2e8 x 64 rows, k = 500, 284.25 ms
    e = bench.roofline_entry("objective_kernel", "simt", 200_000_000, 64, 500.0, 284.25,
                             6785.9, "measured", None)
    assert e["bound"] == "alu" and e["unit"] == "TFLOP/s"
    assert e["algorithmic_flops_per_launch"] == pytest.approx(1.28e13)
    assert e["achieved"] == pytest.approx(1.28e13 / 0.28425 / 1e12, rel=1e-12)
    assert e["frac"] == pytest.approx(0.559, abs=1e-3)


def test_crossover_of_the_cuda_core_form():
    # HBM time 4 n d / B against FMA time 2 n k d / F: the FMAs bind once
    # k > 2 F / B (F in flop/s, B in byte/s), about 23.7 here
    kx = 2 * bench.ALU_PEAK_TFLOPS * 1e12 / (6785.9e9) / 1.0
    assert 23 < kx / 1.0 < 24.5
    lo = bench.roofline_entry("objective_kernel", "simt", 10**7, 16, 23.0, 0.1, 6785.9, "m", None)
    hi = bench.roofline_entry("objective_kernel", "simt", 10**7, 16, 25.0, 0.1, 6785.9, "m", None)
    assert lo["bound"] == "hbm" and hi["bound"] == "alu"


def test_split_bf16_form_at_large_k_is_tensor_bound():
    # the large workload's split-BF16 objective: 2e8 x 64 rows, k = 500 --
    # 1.28e13 flops at a third of the sustained BF16 rate (three BF16
    # products per FP32 product) take longer than 51.2 GB at the HBM rate
    e = bench.roofline_entry("tcb_objective_kernel", "split_bf16", 200_000_000, 64, 500.0, 72.0,
                             6791.7, "measured", None)
    peak, src = bench.tensor_peak("split_bf16")
    assert e["bound"] == "tensor" and e["unit"] == "TFLOP/s" and e["peak"] == peak
    assert "/ 3" in src
    assert e["achieved"] == pytest.approx(1.28e13 / 0.072 / 1e12, rel=1e-12)
    assert e["frac"] == pytest.approx(e["achieved"] / peak, rel=1e-12)


def test_tensor_peaks_of_the_forms():
    bf16 = bench.tensor_peak("split_bf16")[0] * 3
    assert bench.tensor_peak("tf32")[0] == pytest.approx(bf16 * 1.1 / 2.25)
    assert bench.tensor_peak("split_tf32")[0] == pytest.approx(bf16 * 1.1 / 2.25 / 3)
