"""Host logic of the benchmark (no GPU): the work counts behind every reported
rate, the configuration numbers, and the roofline denominators.

The counts are checked against values worked out by hand from the kernels'
launch shapes:
- FP64 solve: 8 flops per complex multiply-add, D^3/6 for the factorisation
  and (1 + 2 refine) C D^2 for the C basis right-hand sides;
- tensor-core covariance, stacked form (D rounded up to 8, D8 <= 64): two
  M = 128 MMAs of NA = G D8 (rounded up to 16) columns per K step, G =
  64 // D8 systems per tile; split form (D8 > 64): four such MMAs, one
  system per tile;
- tensor-core apply: 128 x NP x 2D real MACs per 128-cell tile, NP = 2 S
  weight rows per block in the tile, rounded up to 16.
"""
import json
import os

import pytest

import bench
from paper_2203_06233_gb300 import synth


def _kt():
    return {"doppler": 1.0, "covariance": 1.0, "solve": 1.0, "apply": 1.0}


def test_solve_flops_counts_the_basis_right_hand_sides():
    spec = synth.large_cpi()                      # C32 T4 (D = 128), K512, NB 128
    per = 8.0 * (128 ** 3 / 6.0 + 3 * 32 * 128 ** 2)
    assert bench.solve_flops(spec) == pytest.approx(512 * 128 * per)
    assert bench.solve_flops(spec) == pytest.approx(1.0079e12, rel=1e-4)
    # the explicit steering table solves all S vectors and normalises them in FP64
    per_s = 8.0 * (128 ** 3 / 6.0 + 3 * 64 * 128 ** 2) + 4.0 * 64 * 128
    assert bench.solve_flops(spec, separable=False) == pytest.approx(512 * 128 * per_s)


@pytest.mark.parametrize("name,prec,cov_mac", [
    # split form, D = 128: 4 x 128 x 128 columns x 256 cells x 65536 systems x 3 products
    ("large", 3, 4 * 128 * 128 * 256 * 65536 * 3),
    # stacked form, D = 64: G = 1, NA = 64; 2 x 128 x 64 x 128 cells x 32768 systems x 6
    ("mixed", 1, 2 * 128 * 64 * 128 * 32768 * 6),
    # stacked form, D = 12: D8 = 16, G = 4, NA = 64; 16384 systems in 4096 tiles of 64 cells
    ("standard", 1, 2 * 128 * 64 * 64 * 4096 * 6),
])
def test_tensor_core_covariance_issued_macs(name, prec, cov_mac):
    spec = bench.workload_spec(0, name)
    pk = {"hbm_gbs": 1.0, "bf16_tflops": 1.0, "fp64_tflops": 1.0, "fp32_tflops": 1.0}
    used = {"covariance": "tensor cores", "apply": "tensor cores"}
    k = bench.kernel_figures(spec, prec, _kt(), pk, used=used)
    # 1 ms and a peak of 1 TFLOP/s (fp16 / bf16; TF32 at half): frac = 2 MACs / 1e9
    assert k["covariance"]["bound"] == "tensor"
    assert k["covariance"]["frac"] == pytest.approx(2.0 * cov_mac / 1e9)
    C, P, K, R, T, B, S = spec.dims()
    D = C * T
    nprod = 6 if prec == 1 else 3
    useful = 2.0 * 4 * D * D * B * K * (R // B) * nprod
    assert k["covariance"]["useful_tflops"] == pytest.approx(useful / 1e9)
    if D in (64, 128):   # one system fills the tile: nothing issued is thrown away
        assert k["covariance"]["issued_tflops"] == pytest.approx(k["covariance"]["useful_tflops"])


def test_tensor_core_apply_issued_macs():
    spec = synth.large_cpi()                      # B = 256 -> one block per 128-cell tile, NP = 128
    pk = {"hbm_gbs": 1.0, "bf16_tflops": 1.0, "fp64_tflops": 1.0, "fp32_tflops": 1.0}
    k = bench.kernel_figures(spec, 3, _kt(), pk, used={"covariance": "tensor cores",
                                                       "apply": "tensor cores"})
    mac = 128 * 128 * 2 * 128 * 512 * (32768 // 128) * 3
    assert k["apply"]["frac"] == pytest.approx(2.0 * mac / 1e9)


def test_steps_the_autotuner_kept_on_fp32_are_reported_against_the_fp32_bounds():
    spec = synth.standard_cpi()
    pk = {"hbm_gbs": 1.0, "bf16_tflops": 1.0, "fp64_tflops": 1.0, "fp32_tflops": 1.0}
    k = bench.kernel_figures(spec, 1, _kt(), pk, used={"covariance": "FP32 error-free", "apply": "FP32"})
    assert k["covariance"]["bound"] == "alu" and "fp32_instr" in k["covariance"]
    assert k["apply"]["bound"] == "alu" and "fp32_flops" in k["apply"]
    k = bench.kernel_figures(spec, 1, _kt(), pk, used={"covariance": "FP32 error-free",
                                                       "apply": "tensor cores"})
    assert k["covariance"]["bound"] == "alu" and k["apply"]["bound"] == "tensor"


def test_configuration_numbers_name_the_workloads():
    assert bench.CONFIG_WORKLOADS == {2: "standard", 3: "mixed", 4: "batch", 5: "large"}
    for n, name in bench.CONFIG_WORKLOADS.items():
        if name != "batch":
            assert name in synth.WORKLOADS
    assert bench.workload_spec(0, "large").dims() == (32, 512, 512, 32768, 4, 256, 64)
    assert bench.workload_spec(0, "mixed").dims() == (16, 256, 256, 16384, 4, 128, 32)
    assert bench.workload_spec(0, "standard").dims() == (4, 128, 256, 4096, 3, 64, 16)


def test_peaks_come_from_the_measured_file_when_present():
    p = bench.peaks()
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            m = json.load(f)
        assert p["src"] == "measured" and p["hbm_gbs"] == float(m["hbm_gbs"])
        assert p["bf16_tflops"] == float(m["bf16_tflops"])
    else:
        assert p["src"] == "fallback"
    # FP64 and FP32 from unit counts at the maximum clock
    assert p["fp64_tflops"] == pytest.approx(152 * 2 * 2 * 2.070e9 / 1e12)
    assert p["fp32_tflops"] == pytest.approx(152 * 128 * 2 * 2.070e9 / 1e12)
