"""Host arithmetic of bench.py on CPU: the nominal flop model behind the reported roofline
fraction, the derived FP32 peak, the executed-flop count, the bytes of the lifting roofline and
the kernel-source key under which the measured DRAM traffic is reported."""
import json
import os

import pytest

import bench
import lfa_workloads as W

# Nominal totals per workload, worked out by hand to three digits: Golub-Van Loan dense SVD counts
# (values 4MN^2 - 4N^3/3, values+vectors 14MN^2 + 8N^3, M >= N) times 4 for complex arithmetic,
# plus 4 c_out c_in k^2 for the symbol, over the half-grid frequencies; and the number of
# singular values n m r per layer.
NOMINAL = [
    ("conv4_k3_n8", True, 2.11e5, 256),
    ("conv64_k3_n32", True, 1.19e10, 65536),
    ("conv64_k3_n32", False, 1.51e9, 65536),
    ("resnet18_body", False, 2.28e11, 1417472),
    ("reg4_c128_n32", True, 3.82e11, 524288),
    ("conv512_k3_n64", True, 2.42e13, 2097152),
    ("stem3to64_k7_n224", True, 1.78e9, 150528),
    ("paper_c16_k3_n256", False, 1.73e9, 1048576),
]


@pytest.mark.parametrize("wl,vectors,flops,sigmas", NOMINAL)
def test_nominal_flops_and_sigma_counts(wl, vectors, flops, sigmas):
    layers = W.layers(wl)
    assert abs(sum(bench.layer_flops(l, vectors) for l in layers) / flops - 1) < 0.005
    assert sum(l.n_sigma for l in layers) == sigmas


def test_nominal_count_of_the_benchmark_layer_exactly():
    l = W.layers("conv64_k3_n32")[0]
    # 32 x 32 torus: (1024 + 4) / 2 = 514 half-grid symbols of 64 x 64
    assert bench.layer_flops(l, True) == 514 * (4 * 22 * 64 ** 3 + 4 * 64 * 64 * 9)
    assert bench.layer_flops(l, False) == pytest.approx(514 * (4 * (4 - 4 / 3) * 64 ** 3 + 4 * 64 * 64 * 9))


def test_rectangular_and_strided_symbols_use_the_larger_side_as_rows():
    stem = W.Layer(c_out=64, c_in=3, kh=7, kw=7, n=8, m=8)
    F_h = (64 + 4) // 2
    assert bench.layer_flops(stem, False) == pytest.approx(
        F_h * (4 * 64 * 3 * 49 + 4 * (4 * 64 * 9 - 4 * 27 / 3)))
    strided = W.Layer(c_out=16, c_in=8, kh=3, kw=3, n=8, m=8, sh=2, sw=2)   # symbol 16 x 32
    assert bench.layer_flops(strided, True) == pytest.approx(
        F_h * (4 * 16 * 8 * 9 + 4 * (14 * 32 * 16 ** 2 + 8 * 16 ** 3)))


def test_fp32_peak_is_the_unit_count_times_the_clock():
    assert bench.fp32_peak_tflops() == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)


def test_executed_flops_counts_dots_and_rotations():
    l = W.layers("conv64_k3_n32")[0]
    info = {"sweeps": 10 * 514, "rotations": 1000}
    dots = 10 * 514 * (64 * 63 / 2) * 16 * 64      # 3 complex dots over 64 rows per pair
    assert bench.executed_flops([l], info, True) == pytest.approx(dots + 1000 * 24 * (64 + 64))
    assert bench.executed_flops([l], info, False) == pytest.approx(dots + 1000 * 24 * 64)


def test_lifting_bytes_and_pairs():
    l = W.layers("conv64_k3_n32")[0]
    assert bench.lift_bytes_per_pair(l) == 8 * (64 + 64) * 32 * 32
    assert bench.lift_pairs(l) == 512                               # 512 MiB, more than L2
    s = W.Layer(c_out=16, c_in=8, kh=3, kw=3, n=8, m=8, sh=2, sw=2)
    assert bench.lift_bytes_per_pair(s) == 8 * (16 * 64 + 8 * 16 * 16)   # v_hat on the 16 x 16 input
    tiny = W.layers("conv4_k3_n8")[0]
    assert bench.lift_pairs(tiny) == tiny.F * tiny.r                # capped at every pair


def test_traffic_is_reported_only_under_the_kernel_source_it_was_measured_on(tmp_path, monkeypatch):
    os.makedirs(tmp_path / "profiles")
    with open(tmp_path / "profiles" / "traffic.json", "w") as fh:
        json.dump({"conv64_k3_n32": {"bytes_per_launch": 322816, "kernel_sha16": "aaaa"}}, fh)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_sha16", lambda: "aaaa")
    assert bench.measured_traffic("conv64_k3_n32") == 322816
    assert bench.measured_traffic("resnet18_body") is None
    monkeypatch.setattr(bench, "kernel_sha16", lambda: "bbbb")
    assert bench.measured_traffic("conv64_k3_n32") is None


def test_blocked_route_traffic_scales_with_the_launch_gram_count(tmp_path, monkeypatch):
    """A capture on a smaller case of the blocked route gives bytes per block-pair Gram; the bench
    line's traffic is that times its own launch's Gram count, and null without the count."""
    os.makedirs(tmp_path / "profiles")
    with open(tmp_path / "profiles" / "traffic.json", "w") as fh:
        json.dump({"conv512_k3_n64": {"bytes_per_gram": 1000.0, "kernel_sha16": "aaaa"}}, fh)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_sha16", lambda: "aaaa")
    assert bench.measured_traffic("conv512_k3_n64", {"tc_grams": 2500}) == 2.5e6
    assert bench.measured_traffic("conv512_k3_n64") is None
    monkeypatch.setattr(bench, "kernel_sha16", lambda: "bbbb")
    assert bench.measured_traffic("conv512_k3_n64", {"tc_grams": 2500}) is None

