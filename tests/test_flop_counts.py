"""The numerator of the FP64 roofline: flops per interior point and RK4
stage. The oracle counts the operations of its own literal code with a
counting scalar (add/sub/mul/div = 1, no fused operations). These tests pin
that counter to counts derived by hand from the stencil definitions it
evaluates, pin the composition of the per-point total the benchmark uses,
and set it beside the paper's own figure for the right-hand side. The
last test pins the HBM side: the algorithmic bytes per point and stage."""
import os
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.mark.parametrize("order", [4, 8])
def test_stencil_counts_by_hand(order):
    c = oracle.flop_counts(order)
    H = order // 2          # pairs of the centered stencils
    r = order // 2 + 1      # Kreiss-Oliger radius
    n_up = order + 1        # points of the lopsided upwind stencil
    # first derivative: H subtractions u_a - u_-a, H weight products, H - 1 adds, / h
    assert c["first"] == H + H + (H - 1) + 1
    # second derivative: per pair u_a + u_-a - 2 u_0 (add, mul, sub) and its weight,
    # H - 1 adds, h * h and the division
    assert c["second"] == 4 * H + (H - 1) + 2
    # mixed derivative as the tensor product: per (a, b) three subtractions, the
    # weight product c_a c_b and its product with the difference; H^2 - 1 adds,
    # h h' and the division
    assert c["mixed_tensor"] == 5 * H * H + (H * H - 1) + 2
    # upwind along one axis, both one-sided sums: 2 n products and 2 (n - 1) adds,
    # two divisions by h, (beta +- |beta|) / 2 (2 x (add, mul)), bp dp + bm dm (3)
    assert c["upwind_dir"] == 2 * n_up + 2 * (n_up - 1) + 2 + 4 + 3
    # Kreiss-Oliger per variable: per axis 2r + 1 products, 2r adds, / h; two adds
    # across the axes and the overall factor
    assert c["ko_var"] == 3 * ((2 * r + 1) + 2 * r + 1) + 2 + 1


@pytest.mark.parametrize("order", [4, 8])
def test_gather_is_the_sum_of_its_stencils(order):
    """The oracle's whole gather equals its stencils added up: 54 first
    derivatives (it evaluates d_k gt_ij for all nine (i, j), three of them
    twice), 33 diagonal and 33 mixed second derivatives, 72 upwinded
    directions and 2 adds per variable to sum them; nothing else."""
    c = oracle.flop_counts(order)
    assert c["gather_rhs"] == (54 * c["first"] + 33 * c["second"] + 33 * c["mixed_tensor"]
                               + 72 * c["upwind_dir"] + 24 * 2)


def test_algebra_count_does_not_depend_on_the_order():
    assert oracle.flop_counts(4)["rhs_algebra"] == oracle.flop_counts(8)["rhs_algebra"]
    assert oracle.flop_counts(4)["constraints_algebra"] == oracle.flop_counts(8)["constraints_algebra"]


def test_benchmark_total_from_pinned_parts():
    import bench
    c = oracle.flop_counts(8)
    f = bench.algorithmic_flops(8)
    # 45 first derivatives (the 9 repeated ones left out), 33 second, 33 mixed
    # as first-derivative stencils over shared first derivatives, 72 upwind
    # directions summed per variable
    gather = 45 * c["first"] + 33 * c["second"] + 33 * c["first"] + 72 * c["upwind_dir"] + 48
    assert f["gather"] == gather
    assert f["rhs"] == gather + c["rhs_algebra"]
    assert f["ko"] == 24 * (c["ko_var"] + 1)
    assert f["rk"] == 24 * 4  # acc += b dt k and ynext = y0 + c dt k: two multiply-adds
    assert f["total"] == f["rhs"] + f["ko"] + f["rk"]
    assert f["total"] == 9834


def test_rhs_count_beside_the_paper():
    """The paper quotes about 7900 flops per grid point for one evaluation of
    the BSSN right-hand side at 8th order (Sec. 1.1). The count here, for
    the same system written out independently, is within 5% of it."""
    import bench
    rhs = bench.algorithmic_flops(8)["rhs"]
    assert abs(rhs / 7900 - 1) < 0.05, rhs


def test_stage_bytes_model():
    """The HBM side of the rooflines: the algorithmic bytes per interior
    point of one fused RK4 stage, counted array by array from what the stage
    must touch once (RK4 in the y0 / accumulator form: stage 0 writes the
    accumulator without reading it, stage 3 reads it without writing it),
    and their four-stage means, which the benchmark divides by the stage
    time."""
    import bench
    d, f = 8, 4  # bytes of a double and of a float
    nv, nm, H = 24, 11, 4  # variables, variables with mixed derivatives, 8th-order pairs
    rk = [nv * d * (2 + (s > 0) + (s < 3)) for s in range(4)]  # y0, ynext, acc read, acc written
    assert rk == [576, 768, 768, 576]
    fp64 = [nv * d + 2 * nm * H * d + x for x in rk]  # stage input, x/y difference tables
    fp32 = [nv * f + 2 * nm * f + d + x for x in rk]  # single-precision input, D_x/D_y tables, W
    for s in range(4):
        assert bench.stage_bytes("fp64", s) == fp64[s]
        assert bench.stage_bytes("fp32", s) == fp32[s]
        # inside bssn_rk4_step stages 0..2 also write the next single-precision input
        assert bench.stage_bytes("fp32", s, whole_step=True) == fp32[s] + (nv * f if s < 3 else 0)
    assert bench.mean_stage_bytes("fp64") == 1568
    assert bench.mean_stage_bytes("fp32") == 864
    # 4th order: half the difference-table pairs
    assert bench.stage_bytes("fp64", 1, order=4) == fp64[1] - 2 * nm * 2 * d
