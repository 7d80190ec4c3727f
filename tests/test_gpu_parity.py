"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Small cases (N = 256..301, several assembly tiles plus a ragged tail) are compared
element by element; the large configurations (N = 4096, 16384) on entries the oracle
computes one by one and on residual properties that hold at any size.
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import bem_oracle as O
from paper_2210_08580_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ENTRY_TOL = 1e-13      # |X_gpu - X_orc| <= ENTRY_TOL * max|X_orc|  (matrix entries)
SOLVE_TOL = 1e-10      # FP64 path: relative current error against the oracle
RESID_TOL = 1e-10      # relative residual of the solve on every configuration


@pytest.fixture(scope="module")
def B():
    from paper_2210_08580_gb300 import bem
    bem.load_library()
    return bem


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _np(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def star301():
    v, _, _ = I.equal_chord_mesh(I.cos_star(1.0, 0.3, 5), 301)
    k = 2.0
    return v, k, O.assemble(v, k, "SWD")


@pytest.fixture(scope="module")
def star301_solution(star301):
    v, k, mats = star301
    ang = I.planewave_angles(6)
    f = O.rhs_planewave(v, k, ang)
    h2 = O.rhs_planewave_h(v, k, ang)
    return dict(ang=ang, f=f, h2=h2,
                efie=O.filtered_solve_projected(mats, v, f, 20, 1e-10),
                efie_t=O.filtered_solve_projected(mats, v, f, 20, 1e-4),
                cfie=O.filtered_solve_projected(mats, v, f, 20, 1e-10, alpha=0.5, h2=h2),
                nokernel=O.filtered_solve_projected(mats, v, f, 20, 1e-10, include_kernel=False))


def _solver(B, v, k, ops="SW", **kw):
    s = B.Solver(device=0, **kw)
    s.assemble(_cuda(v), k, ops=ops)
    return s


# ------------------------------------------------------------------ assembly


@pytest.mark.parametrize("ops", ["SWD", "SW"])
def test_assembly_matches_oracle(B, star301, ops):
    v, k, mats = star301
    s = _solver(B, v, k, ops)
    for op in ops:
        g = _np(s.matrix(op))
        assert _rel(g, mats[op]) <= ENTRY_TOL, (op, _rel(g, mats[op]))
    s.close()


def test_assembly_tile_edges_agree(B, star301):
    """bem_options.asm_tile: S and N from tiles of edge 15, 23 and 31 (ragged tails at
    N = 301) all match the oracle, and each other up to the summation order of entries that
    a diagonal tile computes directly and another edge takes from the mirror; any other edge
    is refused at handle creation."""
    v, k, mats = star301
    got = {}
    for T in (15, 23, 31):
        s = _solver(B, v, k, "SW", tiles={"asm_tile": T})
        got[T] = {op: _np(s.matrix(op)) for op in "SW"}
        s.close()
        for op in "SW":
            assert _rel(got[T][op], mats[op]) <= ENTRY_TOL, (T, op, _rel(got[T][op], mats[op]))
    for T in (15, 23):
        for op in "SW":
            assert _rel(got[T][op], got[31][op]) <= 1e-14, (T, op)
    with pytest.raises(B.BemError):
        B.Solver(device=0, tiles={"asm_tile": 16})


@pytest.mark.parametrize("k", [12.0, 24.0])
def test_assembly_bessel_regimes(B, k):
    """k r up to ~24 (Miller recurrence) and ~48 (Hankel asymptotics) on a circle."""
    N = 512
    v = I.regular_polygon(N)
    s = _solver(B, v, k, "SWD")
    rng = np.random.default_rng(3)
    rows = rng.integers(0, N, 120)
    cols = rng.integers(0, N, 120)
    rows[:8] = np.arange(8); cols[:8] = (np.arange(8) + np.array([0, 1, 2, 3, 256, 255, 511, 100])) % N
    ref = O.assemble_entries(v, k, rows, cols, "SWD")
    for op in "SWD":
        g = _np(s.matrix(op))
        scale = np.max(np.abs(g))
        err = np.max(np.abs(g[rows, cols] - ref[op])) / scale
        assert err <= ENTRY_TOL, (op, k, err)
    s.close()


# ------------------------------------------------------------------ rhs, filter, compression, solve


def test_rhs_matches_oracle(B, star301, star301_solution):
    v, k, mats = star301
    sol = star301_solution
    s = _solver(B, v, k, "SW")
    f, vv = s.rhs_planewave(_cuda(sol["ang"]), want_f=True)
    assert _rel(_np(f).T, sol["f"]) <= 1e-13
    assert _rel(_np(vv).T, sol["efie"]["vx"]) <= 1e-12
    s.close()


def test_filter_block_matches_oracle(B, star301, star301_solution):
    v, k, _ = star301
    ref = star301_solution["efie"]
    s = _solver(B, v, k, "SW")
    s.filter_apply(41)
    Bg = _np(s.matrix("B"))
    assert Bg.shape == ref["B"].shape
    assert _rel(Bg, ref["B"]) <= 1e-12, _rel(Bg, ref["B"])
    s.close()


def test_compression_and_solve_match_oracle(B, star301, star301_solution):
    v, k, _ = star301
    sol = star301_solution
    for key, tol in (("efie", 1e-10), ("efie_t", 1e-4)):
        ref = sol[key]
        s = _solver(B, v, k, "SW")
        s.filter_apply(41)
        r = s.compress(tol)
        sig = _np(s.matrix("sigma"))
        assert np.max(np.abs(sig - ref["sigma"])) <= 1e-12 * ref["sigma"][0]
        assert abs(r - ref["rank"]) <= 1
        s.factor()
        vv = s.rhs_planewave(_cuda(sol["ang"]))
        x, it, res = s.solve(vv, report=True)
        assert res <= 1e-13
        xg = _np(x).T
        if r == ref["rank"]:
            assert _rel(xg, ref["x"]) <= SOLVE_TOL, (key, _rel(xg, ref["x"]))
        else:
            assert _rel(xg, ref["x"]) <= 10 * tol
        s.close()


def test_cfie_matches_oracle(B, star301, star301_solution):
    v, k, _ = star301
    ref = star301_solution["cfie"]
    s = _solver(B, v, k, "SWD")
    s.filter_apply(41, alpha=0.5)
    assert _rel(_np(s.matrix("B")), ref["B"]) <= 1e-12
    assert s.compress(1e-10) == ref["rank"]
    s.factor()
    x = s.solve(s.rhs_planewave(_cuda(star301_solution["ang"])))
    assert _rel(_np(x).T, ref["x"]) <= SOLVE_TOL
    assert abs(s.info()["beta"] - 0.5) < 1e-15
    s.close()


def test_literal_filter_without_kernel_mode(B, star301, star301_solution):
    v, k, _ = star301
    ref = star301_solution["nokernel"]
    s = _solver(B, v, k, "SW", include_kernel_mode=False)
    s.filter_apply(41)
    assert s.compress(1e-10) == ref["rank"]
    s.factor()
    x = s.solve(s.rhs_planewave(_cuda(star301_solution["ang"])))
    assert _rel(_np(x).T, ref["x"]) <= SOLVE_TOL
    s.close()


def test_backward_is_the_adjoint_solve(B, star301):
    v, k, _ = star301
    s = _solver(B, v, k, "SW")
    s.filter_apply(41)
    s.compress(1e-10)
    s.factor()
    rng = np.random.default_rng(1)
    g = _cuda(rng.standard_normal((5, v.shape[0])) + 1j * rng.standard_normal((5, v.shape[0])))
    lam = s.solve_backward(g)
    U, Vh = s.matrix("U"), s.matrix("Vh")
    beta = s.info()["beta"]
    # (beta I + U V^H)^H lam = g
    A_H_lam = beta * lam.T + Vh.conj().T @ (U.conj().T @ lam.T)
    assert float((A_H_lam - g.T).abs().max() / g.abs().max()) <= 1e-13
    s.close()


def test_mie_circle_c1(B):
    """C1: unit circle, N = 256, k = 1, n = 65, tol 1e-10, 16 plane waves."""
    N, k, M, nrhs = 256, 1.0, 32, 16
    v = I.regular_polygon(N)
    ang = I.planewave_angles(nrhs)
    s = _solver(B, v, k, "SW")
    s.filter_apply(2 * M + 1)
    s.compress(1e-10)
    s.factor()
    x = _np(s.solve(s.rhs_planewave(_cuda(ang)))).T
    mats = O.assemble(v, k, "SW")
    ref = O.filtered_solve_projected(mats, v, O.rhs_planewave(v, k, ang), M, 1e-10)
    assert _rel(x, ref["x"]) <= SOLVE_TOL
    G = O.gram(v)
    th = 2 * math.pi * np.arange(N) / N
    for w in range(nrhs):
        jm = O.mie_current(k, 1.0, th, ang[w])
        assert O.g_norm(G, x[:, w] - jm)[0] / O.g_norm(G, jm)[0] < 1e-4
    s.close()


# ------------------------------------------------------------------ large configurations
#
# The oracle's block route (tests/golden/make_goldens.py, CPU only) stored, for 16 of each
# configuration's plane waves, the compressed and uncompressed filtered solutions and the
# preconditioned right-hand side at 256 seeded rows, the singular values, the rank and the
# condition number kappa of the filtered operator.  The GPU solutions are compared with them
# element by element, on both paths, with the tolerances of the method's statement:
# FP64 path <= 1e-10 (<= 1e-13 kappa above kappa = 1e3), mixed path <= 1e-8 (<= 1e-11 kappa
# above kappa = 1e3), ranks equal up to one at sigma_r ~ tol sigma_1.

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    with np.load(os.path.join(GOLDEN, name + ".npz")) as z:
        return {key: z[key] for key in z.files}


U64 = 2.0 ** -53


def solution_tolerance(prec, kappa):
    """The stated bars (1e-10 FP64, 1e-8 mixed), loosened with the filtered operator's
    condition number above kappa = 1e3 (1e-13 kappa, 1e-11 kappa)."""
    if prec == "fp64":
        return 1e-10 if kappa <= 1e3 else 1e-13 * kappa
    return 1e-8 if kappa <= 1e3 else 1e-11 * kappa


def _entries_match_oracle(s, v, k, rows, cols, ops="SW"):
    ref = O.assemble_entries(v, k, rows, cols, ops)
    for op in ops:
        g = s.matrix(op)
        scale = float(g.abs().max())
        got = _np(g[torch.as_tensor(rows).cuda(), torch.as_tensor(cols).cuda()])
        err = np.max(np.abs(got - ref[op])) / scale
        assert err <= ENTRY_TOL, (op, k, err)
        del g


def _compare_with_golden(B, v, gold, prec, check_entries=None):
    """Runs the whole path on the GPU for the golden's 16 plane waves and compares the
    right-hand side, singular values, rank and solution with the oracle's."""
    k, M, tol = float(gold["k"]), int(gold["M"]), float(gold["tol"])
    kappa = float(gold["kappa"])
    rows = gold["rows"]
    # the mixed path refines to the relative residual the method's precision configuration
    # states (1e-8); the FP64 path needs no refinement
    s = B.Solver(device=0, prec=prec, refine_rtol=1e-8)
    s.assemble(_cuda(v), k, ops="SW")
    if check_entries is not None:
        _entries_match_oracle(s, v, k, *check_entries)
    vv = s.rhs_planewave(_cuda(gold["angles"]))
    s.filter_apply(2 * M + 1)
    r = s.compress(tol)
    sig = _np(s.matrix("sigma"))
    s.factor()
    x, it, res = s.solve(vv, report=True)
    xs = _np(x).T[rows]
    vs = _np(vv).T[rows]
    s.close()
    rhs_err = _rel(vs, gold["vx"])
    sig_err = float(np.max(np.abs(sig - gold["sigma"])) / gold["sigma"][0])
    tol_x = solution_tolerance(prec, kappa)
    if r == int(gold["rank"]):
        x_err = _rel(xs, gold["x"])
    else:
        # A11: at sigma_r ~ tol sigma_1 the ranks may differ by one; both sides then lie
        # within the truncation error of the uncompressed filtered solution
        x_err = _rel(xs, gold["x_full"])
        tol_x = max(tol_x, 10 * tol * kappa)
    # u c_rowsum: how far rounding N's entries to FP64 can move its row sums (relative), which
    # at low k carry the constant mode; the library restores them exactly from the assembly
    print(f"{prec} N={len(v)} k={k:g}: kappa={kappa:.3g} u*c_rowsum={U64 * float(gold['c_rowsum']):.2g} "
          f"rank gpu/oracle={r}/{int(gold['rank'])} "
          f"x err={x_err:.2e} (tol {tol_x:.1e}) v err={rhs_err:.2e} sigma err={sig_err:.2e} resid={res:.1e}")
    assert abs(r - int(gold["rank"])) <= 1
    assert x_err <= tol_x, (prec, k, x_err, tol_x, kappa)
    assert rhs_err <= (1e-12 if prec == "fp64" else 5e-10), (prec, rhs_err)
    assert sig_err <= (1e-11 if prec == "fp64" else 1e-9), (prec, sig_err)
    assert res <= (RESID_TOL if prec == "fp64" else 1e-8)
    return dict(kappa=kappa, x_err=x_err, rank=r)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("k", [1e-3, 1e-2, 1e-1, 1.0, 5.0])
def test_c2_star_4096_against_oracle(B, k, prec):
    """C2: r = 1 + 0.3 cos 5t, N = 4096, n = 201, tol 1e-10 (16 of the 256 plane waves),
    every wavenumber of the low-frequency sweep, both paths, against the oracle."""
    N = 4096
    v, _, _ = I.equal_chord_mesh(I.cos_star(1.0, 0.3, 5), N)
    gold = _golden(f"c2_star_n4096_k{k:g}")
    ent = None
    if prec == "fp64":
        rng = np.random.default_rng(int(k * 1000) + 7)
        rows = np.concatenate([rng.integers(0, N, 48), np.arange(8)])
        cols = np.concatenate([rng.integers(0, N, 48), (np.arange(8) + np.array([0, 1, 2, 5, 2048, 4095, 3, 1])) % N])
        ent = (rows, cols)
    _compare_with_golden(B, v, gold, prec, ent)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_c3_random_star_16384_against_oracle(B, prec):
    """C3 at full size (random 8-harmonic star of seed 0, N = 16384, k = 2, n = 201,
    tol 1e-10; 16 of the 1024 plane waves): sampled entries, right-hand side, singular
    values, rank and solution against the oracle, on the FP64 and the mixed path."""
    N = 16384
    v, _, _ = I.equal_chord_mesh(I.random_star(0), N)
    gold = _golden("c3_random_star0_n16384")
    ent = None
    if prec == "fp64":
        rng = np.random.default_rng(11)
        rows = np.concatenate([rng.integers(0, N, 40), np.arange(6)])
        cols = np.concatenate([rng.integers(0, N, 40), (np.arange(6) + np.array([0, 1, 2, 8192, 16383, 4])) % N])
        ent = (rows, cols)
    _compare_with_golden(B, v, gold, prec, ent)


# ------------------------------------------------------------------ errors and edge cases


def test_errors_are_reported_not_raised_on_device(B):
    v = I.regular_polygon(64)
    s = B.Solver(device=0)
    with pytest.raises(B.BemError) as e:
        s.filter_apply(15)
    assert e.value.status == 1
    # a mesh too coarse for the wavenumber (k h > 2)
    with pytest.raises(B.BemError) as e:
        s.assemble(_cuda(v), 100.0)
    assert e.value.status == 4
    # unequal chords are a general mesh, not an error
    vb = v.copy()
    vb[3] *= 1.01
    s.assemble(_cuda(vb), 1.0)
    assert s.info()["equal_chord"] == 0
    s.assemble(_cuda(v), 1.0)
    assert s.info()["equal_chord"] == 1
    for bad in (14, 2, 64):
        with pytest.raises(B.BemError):
            s.filter_apply(bad)
    with pytest.raises(B.BemError):
        s.filter_apply(15, alpha=1.0)        # needs D
    s.filter_apply(15)
    with pytest.raises(B.BemError):
        s.factor()                           # compress first
    s.compress(1e-10)
    s.factor()
    x = s.solve(s.rhs_planewave(_cuda(I.planewave_angles(3))))
    assert torch.isfinite(torch.view_as_real(x)).all()
    s.close()


def test_smallest_mesh_and_single_rhs(B):
    N, k = 16, 0.5
    v = I.regular_polygon(N)
    s = _solver(B, v, k, "SW")
    s.filter_apply(7)
    s.compress(0.0)
    s.factor()
    ang = np.array([0.7])
    x = _np(s.solve(s.rhs_planewave(_cuda(ang)))).T
    mats = O.assemble(v, k, "SW")
    ref = O.filtered_solve_projected(mats, v, O.rhs_planewave(v, k, ang), 3, 0.0)
    assert _rel(x, ref["x"]) <= SOLVE_TOL
    s.close()
