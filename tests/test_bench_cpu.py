"""bench.py's roofline arithmetic on made-up per-kernel reports (host logic only): the
dominant kernel, the method's own flop count of the split products (the complex FP64
products they stand for) beside the bf16 emulation count (slice pairs times the real
products), the FP32-operation count of the assembly, and the oracle timing fit."""
import types

import pytest

import bench


def _args(N=16384, nrhs=1024):
    return types.SimpleNamespace(N=N, nrhs=nrhs)


def test_tensor_roofline_of_the_rhs_product_counts_the_method_work():
    rep = {"tc_rhs_SY": (3, 3 * 18.4), "k_assemble": (3, 3 * 16.7), "k_jacobi": (3, 3 * 5.3)}
    roof, rows = bench.roofline(rep, _args(), 201, 201, 6.7e8)
    assert roof["kernel"] == "tc_rhs_SY" and roof["bound"] == "tensor"
    method = 8 * 16384 * 16384 * 1024                       # v = S Y, complex FP64 product
    assert roof["method_flops_per_launch"] == pytest.approx(method)
    assert roof["achieved"] == pytest.approx(method / 18.4e-3 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    emu = roof["emulation"]
    assert emu["slice_pairs"] == 15                        # five slices per operand
    flops = 15 * 2 * 3 * 16384 * 1024 * 16384              # complex x complex: Gauss's three real products
    assert emu["bf16_flops_per_launch"] == pytest.approx(flops)
    assert emu["frac"] == pytest.approx(15 * 0.75 * roof["frac"])
    assert roof["traffic"] == bench.TRAFFIC_BYTES.get("tc_rhs_SY")
    assert [r["kernel"] for r in rows] == ["tc_rhs_SY", "k_assemble", "k_jacobi"]


def test_alu_roofline_of_the_assembly():
    rep = {"k_assemble": (2, 2 * 16.7), "tc_rhs_SY": (2, 2 * 10.0)}
    roof, _ = bench.roofline(rep, _args(), 201, 201, 6.7e8)
    assert roof["kernel"] == "k_assemble" and roof["bound"] == "alu"
    assert roof["ops_per_unit"] == bench.ASM_OPS_PER_POINT and roof["units_per_launch"] == 6.7e8
    assert roof["achieved"] == pytest.approx(6.7e8 * bench.ASM_OPS_PER_POINT / 16.7e-3 / 1e12)
    assert roof["peak"] == pytest.approx(152 * 128 * 2.07e9 / 1e12)


def test_filter_products_count_real_and_complex_parts():
    # Q^T S: the real Fourier basis times a complex operator, two real products per pair;
    # Y N: complex times complex, three (Gauss's form over the Re, Im, Re + Im blocks)
    a = bench.tc_gemm_flops("tc_filter_QtS", 1024, 64, 21, 21, 6)
    b = bench.tc_gemm_flops("tc_filter_YN", 1024, 64, 21, 21, 6)
    assert a == pytest.approx(21 * 2 * 2 * 21 * 1024 * 1024)
    assert b == pytest.approx(1.5 * a)
    assert bench.tc_gemm_flops("k_iir", 1024, 64, 21, 21, 6) is None
    args = _args(N=1024, nrhs=64)
    assert bench.method_flops("tc_filter_QtS", args, 21) == pytest.approx(4 * 21 * 1024 * 1024)
    assert bench.method_flops("tc_filter_YN", args, 21) == pytest.approx(8 * 21 * 1024 * 1024)


def test_filter_pair_reported_together():
    rep = {"tc_rhs_SY": (1, 18.0), "k_assemble": (1, 16.0), "tc_filter_YN": (1, 6.0), "tc_filter_QtS": (1, 3.0)}
    _, rows = bench.roofline(rep, _args(), 201, 201, 6.7e8)
    assert [r["kernel"] for r in rows] == ["tc_rhs_SY", "k_assemble", "tc_filter_YN", "tc_filter_QtS"]


def test_basis_products_of_a_general_mesh():
    """Non-equal-chord mesh: the double-float basis products count their algorithmic flops,
    2 N p^2 per Gram product, 2 N p n for the one Q = X Cf launch per step, N p (p + 1) per
    triangular re-orthonormalisation X R^-1, against the double-float peak derived from the
    FP32 pipe; the one-CTA Cholesky counts p^3 / 3 against one SM."""
    N, p, n, steps = 16384, 411, 201, 3
    basis = {"block": p, "iters": 34, "ncols": n}
    rep = {"k_dgemm_df": (16 * steps, steps * 30.0), "k_dgemm_df_tri": (15 * steps, steps * 20.0),
           "k_chol": (16 * steps, steps * 35.0)}
    _, rows = bench.roofline(rep, _args(N=N), n, 201, 0, basis=basis, nsteps=steps)
    by = {r["kernel"]: r for r in rows}
    g = by["k_dgemm_df"]
    fl = (15 * 2.0 * N * p * p + 2.0 * N * p * n) / 16
    assert g["flops_per_launch"] == pytest.approx(fl)
    assert g["achieved"] == pytest.approx(fl / (30.0e-3 / 16) / 1e12)
    assert g["peak"] == pytest.approx(152 * 128 * 2.07e9 / 1e12 * 2 / bench.DF_OPS_PER_FMA)
    t = by["k_dgemm_df_tri"]
    assert t["flops_per_launch"] == pytest.approx(float(N) * p * (p + 1))
    c = by["k_chol"]
    assert c["flops_per_launch"] == pytest.approx(p ** 3 / 3.0)
    assert c["peak"] == pytest.approx(128 * 2.07e9 / 1e12 * 2 / bench.DF_OPS_PER_FMA)
