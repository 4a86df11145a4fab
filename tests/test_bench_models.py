"""The arithmetic behind bench.py's roofline fields (host logic, no GPU):
padded FFT geometry and folding, the algorithmic bytes of the FFT passes and
of the gather, the exact kernel's operations per pair and its polynomial
length, the tensor-core product's executed operations, and the derived FP32
peak.  Expected values are worked out by hand from the pass-by-pass
description (x pass: data grid in, x-padded grid out; y pass: x-padded in,
xy-padded out; z pass: xy-padded in and out plus the stored spectrum)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2312_02376_gb300 import inputs  # noqa: E402

K2D = 2 * 3.141592653589793 * 0.8
K3D = 2 * 3.141592653589793 * 2.0


def workload(name, D, pdims, k, k0, n, b, nf, N):
    return inputs.Workload(name, D, pdims, k, k0, n, 4, 1, b, nf, 4, "fp32", N)


C2 = workload("helmholtz2d_262k", (1.0, 1.0, 0.5), (0, 1), K2D, (0.3 * K2D, 0.1 * K2D, 0.0), (128, 128, 64), 4,
              (21, 21, 11), 262144)
C5 = workload("helmholtz3d_16m", (1.0, 1.0, 1.0), (0, 1, 2), K3D, (0.2 * K3D, 0.2 * K3D, 0.0), (512, 512, 512), 5,
              (51, 51, 51), 16_000_000)
SPHERES = workload("helmholtz3d_spheres_1m", (1.0, 1.0, 1.0), (0, 1, 2), K3D, (0.2 * K3D, 0.2 * K3D, 0.0),
                   (256, 256, 256), 5, (51, 51, 51), 1_000_000)


class Info:
    """The fields of pim_info that the byte models read."""
    def __init__(self, nnz, corr_mode, lf_tc_boxes=0):
        self.nnz = nnz
        self.corr_mode = corr_mode
        self.lf_tc_boxes = lf_tc_boxes


def test_fft_geometry_pads_to_powers_of_two_and_folds_even_axes():
    # 2n - 1 = 255, 255, 127 -> 256, 256, 128; x and y carry a phase shift
    # (no folding), z is open (even kernel: 0..L/2 kept)
    assert bench.fft_geometry(C2) == ([256, 256, 128], [256, 256, 65])
    # 3D lattice, phase along x and y only: z folds
    assert bench.fft_geometry(C5) == ([1024, 1024, 1024], [1024, 1024, 513])


def test_fft_pass_bytes_of_the_2d_workload():
    # x pass 128*128*64 + 256*128*64 complex64 = 25,165,824 B, twice (forward
    # and inverse); y pass 256*128*64 + 256*256*64 = 50,331,648 B, twice; z
    # pass 2 * 256*256*64 plus the folded spectrum 256*256*65, 101,187,584 B
    assert bench.stage_bytes(C2, Info(0, 3))["fft"] == 2 * 25_165_824 + 2 * 50_331_648 + 101_187_584


def test_fft_pass_bytes_of_the_3d_workload():
    x = (512 ** 3 + 1024 * 512 * 512) * 8
    y = (1024 * 512 * 512 + 1024 * 1024 * 512) * 8
    z = 2 * 1024 * 1024 * 512 * 8 + 1024 * 1024 * 513 * 8
    assert bench.stage_bytes(C5, Info(0, 3))["fft"] == 2 * x + 2 * y + z == 32_220_643_328


def test_gather_bytes_per_entry_and_per_point():
    N, G = 1000, 4096
    base = bench.gather_bytes(Info(0, 3), N, G, 0)
    # compact rows: column 4 B + FP32 head 8 B per entry, 4 B more per double-float entry
    assert bench.gather_bytes(Info(100, 3), N, G, 0, nbig=10) - base == 100 * 12 + 10 * 4
    # FP64 values: 16 B value + 4 B column
    assert bench.gather_bytes(Info(100, 0), N, G, 0, fp64=True) - bench.gather_bytes(Info(0, 0), N, G, 0,
                                                                                     fp64=True) == 100 * 20
    # per point (FP32): stencil start 4, local coordinates 12, permutation 4,
    # sorted source 8, output 8, row split 4; row pointers 8 (N + 1); the grid once
    assert base == (N + 1) * 8 + N * 40 + G * 8


def test_exact_kernel_operations_and_polynomial_length():
    # 18 operations plus 2 x 2 per extra polynomial term
    assert bench.lf_pair_flops(4) == 30 and bench.lf_pair_flops(5) == 34
    # k r at most k (R + 1) h sqrt(3) with R = b + 1 = 6: 0.298 at h = 1/511
    # (terms: x^2/2, x^4/24, x^6/720 = 1e-6, x^8/40320 = 1.6e-9 < 1.5e-8 -> 4),
    # 0.597 at h = 1/255 (x^8/40320 = 4e-7, x^10/3628800 = 1.6e-9 -> 5)
    assert bench.lf_nterm(C5) == 4
    assert bench.lf_nterm(SPHERES) == 5


def test_tensor_core_product_operations():
    # E = 2 (b + 1) + 2 floor(p/2) + p + 1 = 21, KP = 9261 padded to 9280: per box
    # three products of a 256 x 18560 operator by one 18560-row, 6 * 256 * 18560
    r = bench.tc_roofline(C5, Info(0, 3, lf_tc_boxes=72291), 5.0)
    assert r["executed_flops_per_launch"] == 6.0 * 256 * 18560 * 72291
    assert r["useful_complex_flops_per_launch"] == 8.0 * 125 * 21 ** 3 * 72291
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(6.0 * 256 * 18560 * 72291 / 5e-3 / 1e12, rel=1e-3)


def test_fp32_alu_peak():
    assert bench.fp32_alu_peak() == pytest.approx(152 * 128 * 2 * 2.07e9)


def test_correction_modes_match_the_library():
    from paper_2312_02376_gb300 import pim
    assert bench.CORR_MODES == {"fp64": pim.PIM_CORR_FP64, "double_float": pim.PIM_CORR_DOUBLE_FLOAT,
                                "fp32": pim.PIM_CORR_FP32, "compact": pim.PIM_CORR_COMPACT}
    assert set(bench.CORR_TEXT) == set(bench.CORR_MODES.values()) == set(bench.VALUE_BYTES)
    # FP64 values: 16 B per complex value, the double-float split too; complex64 and compact heads 8 B
    assert bench.VALUE_BYTES == {0: 16, 1: 16, 2: 8, 3: 8}
