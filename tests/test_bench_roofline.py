"""The benchmark's per-kernel algorithmic bytes and achieved-bandwidth
arithmetic (host logic, no GPU): the bytes each kernel of the step must move
at the minimum, and the fraction of the measured HBM rate they give over a
kernel's mean launch time."""
import pytest

import bench

N, C = 1000, 64


def test_field_update_moves_e_b_j_in_and_e_b_out_once():
    # 9 values read (E, B, J) and 6 written (E, B) per cell
    assert bench.kernel_bytes("k_yee_fused", N, C, "fp32")[0] == C * 15 * 4
    assert bench.kernel_bytes("k_yee_fused", N, C, "fp64")[0] == C * 15 * 8
    # the in-place passes: B half step reads E, B and writes B; E step reads E, B, J and writes E
    assert bench.kernel_bytes("k_yee_b", N, C, "fp32")[0] == C * 9 * 4
    assert bench.kernel_bytes("k_yee_e", N, C, "fp32")[0] == C * 12 * 4


def test_tile_kernel_and_sort_bytes():
    # FP32-mixed: key + 3 offsets + 3 u + w read, key + 3 offsets + 3 u written;
    # E, B read and J written per cell
    assert bench.kernel_bytes("k_tile_step", N, C, "fp32")[0] == N * 60 + C * 36
    assert bench.kernel_bytes("k_tile_step", N, C, "fp64")[0] == N * 104 + C * 72
    assert bench.kernel_bytes("k_scatter_perm", N, C, "fp32")[0] == N * 8 + C * 4
    assert bench.kernel_bytes("k_scan", N, C, "fp32")[0] == C * 8
    assert bench.kernel_bytes("k_hist", N, C, "fp32")[0] == N * 4 + C * 4
    assert bench.kernel_bytes("k_outsiders", N, C, "fp32") is None


def test_rooflines_divide_bytes_by_the_mean_launch_time():
    # two launches of 1 ms in all: 0.5 ms each
    out = bench.kernel_rooflines({"k_yee_fused": (1.0, 2), "k_outsiders": (0.1, 2), "k_scan": (0.0, 0)},
                                 N, C, "fp32", hbm_gbs=10.0)
    assert set(out) == {"k_yee_fused"}
    r = out["k_yee_fused"]
    assert r["bytes_per_launch"] == C * 60
    assert r["achieved_gbs"] == pytest.approx(C * 60 / 0.5e-3 / 1e9)
    assert r["frac_of_hbm"] == pytest.approx(r["achieved_gbs"] / 10.0)


def test_step_bytes_follow_the_kernels():
    # the whole step: tile kernel, one-pass field update, and a sort of 76 B a particle (FP32-mixed)
    assert bench.step_bytes(N, C, "fp32") == N * 60 + C * 36 + C * 60 + N * 76
    assert bench.step_bytes(N, C, "fp32", sort=False) == N * 60 + C * 36 + C * 60
