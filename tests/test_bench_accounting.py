"""The benchmark's roofline numerators for the 2048 x 1024, 3-field, 2,097,152-
point workload, against the byte and flop counts worked out by hand from their
definitions (what each stage must read and write once; the reference traffic
model 13 N1 N2 c + 16 P / F + s_out P per field at sigma 2)."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


P, F, ROWS = 2_097_152, 3, 2096
C3_F32 = {"N1": 2048, "N2": 2048, "n1": 4096, "n2": 4096, "dtype": 1, "flags": 1, "sigma": 2,
          "w": 7}
C3_F64 = dict(C3_F32, dtype=0, w=14)


def test_stage_bytes_fp32(bench):
    b = bench.stage_bytes(C3_F32, F, P, ROWS)
    # fine rows 2096 x 4096 x 4 B per field and 4-byte values, plus the sorted
    # records (int2 base, two FP32 offsets, int index = 20 B a point)
    assert b["interp"] == 3 * (2096 * 4096 * 4 + P * 4) + P * 20 == 170_131_456
    # reads T (1025 columns x 8 B of the needed rows), writes the real rows
    assert b["phi_pass"] == 3 * (2096 * 1025 * 8 + 2096 * 4096 * 4)
    # coefficient columns m >= 0 plus the Nyquist column (1026 x 8 B a row), T
    # written, and the two deconvolution factor vectors
    assert b["theta_pass"] == 3 * (2048 * 1026 * 8 + 2096 * 1025 * 8) + 8 * 4096
    # lon, colat read twice (fold, scatter), the rank, the sorted records
    assert b["set_points"] == P * 20 + P * 20 + P * 20


def test_model_bytes(bench):
    assert bench.model_bytes(C3_F32, F, P) == 3 * (2048 * 2048 * 8 * 13 + 4 * P) + 16 * P \
        == 1_367_343_104
    assert bench.model_bytes(C3_F64, F, P) == 3 * (2048 * 2048 * 16 * 13 + 8 * P) + 16 * P


def test_interp_flops_fp64(bench):
    # per point and field 2 w (w + 1) for the taps and row sums, per point 4 w^2
    # for the kernel weights
    assert bench.interp_flops(C3_F64, F, P) == P * (3 * 2 * 14 * 15 + 4 * 14 * 14)


def test_df32_interp_ops(bench):
    # w = 14: 7 mirror pairs of Horner chains with 13 steps together (15 FP32
    # instructions each), a product (7) and two sums (11 each): 224 a pair, 7
    # pairs plus u = s^2 (7) for each of x and y; per field 14 rows of 14 Dot2
    # steps (12 each), a renormalisation (3) and one more Dot2 step
    per_point = 2 * (7 * (13 * 15 + 7 + 2 * 11) + 7) + 3 * (14 * (14 * 12 + 3 + 12))
    assert per_point == 10836
    assert bench.df32_interp_ops(C3_F64, F, P) == P * per_point


def test_fft_flops(bench):
    import math
    assert bench.fft_flops(C3_F32, F, ROWS, "theta_pass") == 3 * 1025 * 5.0 * 4096 * 12
    assert bench.fft_flops(C3_F32, F, ROWS, "phi_pass") == 3 * ROWS * 5.0 * 2048 * math.log2(2048)
