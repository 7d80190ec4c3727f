"""Mixed-precision path (split-bf16 tcgen05 products + FP64 refinement) against the CPU
oracle and against the FP64 GPU path.

Bar (the mixed path's accuracy target): the refined mixed solution within 1e-8 of the FP64 reference.
The operator blocks themselves are checked tighter, at the accuracy the split gives."""
import numpy as np
import pytest
import torch

from oracle import bem_oracle as O
from paper_2210_08580_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MIXED_SOLVE_TOL = 1e-8      # relative current error after refinement
# preconditioned RHS v, relative to max: its product S Y keeps 5 of the 6 digit slices
# (35 bits), so its error is a few times 2^-35 (2.9e-11) of max|v| -- measured 1.2e-10 on the
# 301-point star; the solution bar below is the method's accuracy target
MIXED_RHS_TOL = 5e-10
MIXED_BLOCK_TOL = 1e-9      # filtered block B, relative to max: B = Y/g - Q^T/4 cancels ~3 digits


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def B():
    from paper_2210_08580_gb300 import bem
    bem.load_library()
    return bem


@pytest.fixture(scope="module")
def star301_ref():
    v, _, _ = I.equal_chord_mesh(I.cos_star(1.0, 0.3, 5), 301)
    k = 2.0
    mats = O.assemble(v, k, "SWD")
    ang = I.planewave_angles(6)
    f = O.rhs_planewave(v, k, ang)
    h2 = O.rhs_planewave_h(v, k, ang)
    return dict(v=v, k=k, ang=ang,
                efie=O.filtered_solve_projected(mats, v, f, 20, 1e-10),
                cfie=O.filtered_solve_projected(mats, v, f, 20, 1e-10, alpha=0.5, h2=h2))


def test_mixed_blocks_and_solve_match_oracle(B, star301_ref):
    ref = star301_ref["efie"]
    s = B.Solver(device=0, prec="mixed")
    s.assemble(_cuda(star301_ref["v"]), star301_ref["k"], ops="SW")
    vv = s.rhs_planewave(_cuda(star301_ref["ang"]))
    assert _rel(vv.cpu().numpy().T, ref["vx"]) <= MIXED_RHS_TOL
    s.filter_apply(41)
    Bg = s.matrix("B").cpu().numpy()
    assert _rel(Bg, ref["B"]) <= MIXED_BLOCK_TOL, _rel(Bg, ref["B"])
    assert s.compress(1e-10) == ref["rank"]
    s.factor()
    x, it, res = s.solve(vv, report=True)
    assert res <= 1e-10
    assert _rel(x.cpu().numpy().T, ref["x"]) <= MIXED_SOLVE_TOL
    s.close()


def test_rhs_slices_option(B, star301_ref):
    """bem_options.rhs_slices: the right-hand-side product S Y with all six digit slices is
    about two orders more accurate than with the default five (the leading five of the
    same split); both stay inside their tolerances against the oracle."""
    ref = star301_ref["efie"]
    err = {}
    for rs in (5, 6):
        s = B.Solver(device=0, prec="mixed", rhs_slices=rs)
        s.assemble(_cuda(star301_ref["v"]), star301_ref["k"], ops="SW")
        vv = s.rhs_planewave(_cuda(star301_ref["ang"]))
        err[rs] = _rel(vv.cpu().numpy().T, ref["vx"])
        s.close()
    assert err[5] <= MIXED_RHS_TOL, err
    assert err[6] <= 1e-10, err
    assert err[6] < 0.25 * err[5], err


def test_mixed_cfie(B, star301_ref):
    ref = star301_ref["cfie"]
    s = B.Solver(device=0, prec="mixed")
    s.assemble(_cuda(star301_ref["v"]), star301_ref["k"], ops="SWD")
    s.filter_apply(41, alpha=0.5)
    assert _rel(s.matrix("B").cpu().numpy(), ref["B"]) <= MIXED_BLOCK_TOL
    s.compress(1e-10)
    s.factor()
    x = s.solve(s.rhs_planewave(_cuda(star301_ref["ang"])))
    assert _rel(x.cpu().numpy().T, ref["x"]) <= MIXED_SOLVE_TOL
    s.close()


def test_mixed_matches_fp64_c3_16384(B):
    """C3 (N = 16384, k = 2, n = 201, tol 1e-10): mixed-path solution within 1e-8 of the
    FP64 GPU path on the same geometry, with the FP64 residual reported below 1e-10."""
    N, k, M, nrhs = 16384, 2.0, 100, 64
    v, _, _ = I.equal_chord_mesh(I.random_star(0), N)
    ang = _cuda(I.planewave_angles(nrhs))
    xs = {}
    for prec in ("fp64", "mixed"):
        s = B.Solver(device=0, prec=prec)
        s.assemble(_cuda(v), k, ops="SW")
        s.filter_apply(2 * M + 1)
        s.compress(1e-10)
        s.factor()
        vv = s.rhs_planewave(ang)
        x, it, res = s.solve(vv, report=True)
        assert res <= 1e-10, (prec, res)
        xs[prec] = x
        s.close()
    err = float((xs["mixed"] - xs["fp64"]).abs().max() / xs["fp64"].abs().max())
    assert err <= MIXED_SOLVE_TOL, err


def test_refinement_sweeps_recover_a_crude_solve(B, star301_ref):
    """bem_options.solve_slices = 3: the Woodbury solves run on 3 digit slices (about 21
    bits) while the residual products keep all six, so the first iterate misses
    refine_rtol and the FP64-residual refinement (Sec. IV-C solve, mixed path) has to
    sweep; the refined solution meets the same bars as the default path."""
    ref = star301_ref["efie"]
    s = B.Solver(device=0, prec="mixed", solve_slices=3)
    s.assemble(_cuda(star301_ref["v"]), star301_ref["k"], ops="SW")
    s.filter_apply(41)
    assert s.compress(1e-10) == ref["rank"]
    s.factor()
    vv = s.rhs_planewave(_cuda(star301_ref["ang"]))
    x, it, res = s.solve(vv, report=True)
    assert it >= 1, it
    assert res <= 1e-10, res
    assert _rel(x.cpu().numpy().T, ref["x"]) <= MIXED_SOLVE_TOL
    s.close()


def test_refinement_budget_exhausted_reports_not_converged(B, star301_ref):
    """With the crude 3-slice solve and max_refine = 0 the residual stays above
    refine_rtol: solve_many returns BEM_E_NOT_CONVERGED, reports the residual, and leaves
    the unrefined iterate in x (close to the oracle at the 3-slice accuracy)."""
    ref = star301_ref["efie"]
    s = B.Solver(device=0, prec="mixed", solve_slices=3, max_refine=0)
    s.assemble(_cuda(star301_ref["v"]), star301_ref["k"], ops="SW")
    s.filter_apply(41)
    s.compress(1e-10)
    s.factor()
    vv = s.rhs_planewave(_cuda(star301_ref["ang"]))
    x = torch.zeros_like(vv)
    with pytest.raises(B.BemError) as e:
        s.solve(vv, report=True, out=x)
    assert e.value.status == 6                       # BEM_E_NOT_CONVERGED
    assert "residual" in str(e.value)
    err = _rel(x.cpu().numpy().T, ref["x"])
    assert 1e-12 < err <= 1e-3, err
    s.close()
