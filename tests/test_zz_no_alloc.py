"""solve_many_noalloc: the solve for callers that cannot allocate device memory while they
serve requests (stream capture, start-up-reserved memory, foreign allocators).  Its result
must equal solve_many's FP64 result, on consecutive calls that reuse the shared fixed
scratch array.  Collected last so that a stop-at-first-failure run has run everything else."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2210_08580_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12     # relative agreement, as for the other internal-block comparisons


def _solver():
    from paper_2210_08580_gb300 import bem
    v, _, _ = I.equal_chord_mesh(I.cos_star(1.0, 0.3, 5), 301)
    s = bem.Solver(device=0)
    s.assemble(torch.from_numpy(v).cuda(), 2.0, ops="SW")
    s.filter_apply(41)
    s.compress(1e-10)
    s.factor()
    return s


def test_noalloc_matches_solve_many_on_consecutive_calls():
    s = _solver()
    N = s.N
    for seed, nrhs in ((0, 7), (1, 13)):
        rng = np.random.default_rng(seed)
        vv = torch.from_numpy(rng.standard_normal((nrhs, N)) + 1j * rng.standard_normal((nrhs, N))).cuda()
        ref = s.solve(vv)
        x = torch.full_like(vv, float("nan"))
        st = s.L.solve_many_noalloc(s.h, vv.data_ptr(), N, x.data_ptr(), N, nrhs)
        assert st == 0, s.L.bem_last_error(s.h)
        torch.cuda.synchronize()
        err = float((x - ref).abs().max() / ref.abs().max())
        assert err <= TOL, err
    s.close()


def test_noalloc_rejects_requests_beyond_its_scratch():
    s = _solver()
    r = s.info()["r"]
    nrhs = (1 << 18) // r + 1
    vv = torch.zeros((nrhs, s.N), dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(vv)
    st = s.L.solve_many_noalloc(s.h, vv.data_ptr(), s.N, x.data_ptr(), s.N, nrhs)
    assert st == 4
    assert b"262144" in s.L.bem_last_error(s.h)
    s.close()


def test_noalloc_rejects_more_rhs_than_solve_many_accepts():
    """nrhs above 2^24 (solve_many's own limit) is rejected as an invalid argument before
    any work is enqueued; the pointers are never read."""
    s = _solver()
    vv = torch.zeros((1, s.N), dtype=torch.complex128, device="cuda")
    x = torch.zeros_like(vv)
    st = s.L.solve_many_noalloc(s.h, vv.data_ptr(), s.N, x.data_ptr(), s.N, (1 << 24) + 1)
    assert st == 1
    assert b"2^24" in s.L.bem_last_error(s.h)
    s.close()


def test_noalloc_on_a_mixed_handle_matches_the_refined_solve():
    """On a mixed-precision handle the allocation-free call solves with that handle's
    tensor-core-built factors in FP64 and no refinement; its result equals solve_many's
    refined result (which converges to the same operator's inverse) and meets the mixed
    path's 1e-8 bar against the FP64 handle's solution."""
    from paper_2210_08580_gb300 import bem
    v, _, _ = I.equal_chord_mesh(I.cos_star(1.0, 0.3, 5), 301)
    ang = torch.from_numpy(I.planewave_angles(9)).cuda()
    sols = {}
    for prec in ("fp64", "mixed"):
        s = bem.Solver(device=0, prec=prec)
        s.assemble(torch.from_numpy(v).cuda(), 2.0, ops="SW")
        s.filter_apply(41)
        s.compress(1e-10)
        s.factor()
        vv = s.rhs_planewave(ang)
        ref, it, res = s.solve(vv, report=True)
        x = torch.full_like(vv, float("nan"))
        for _ in range(2):
            st = s.L.solve_many_noalloc(s.h, vv.data_ptr(), s.N, x.data_ptr(), s.N, vv.shape[0])
            assert st == 0, s.L.bem_last_error(s.h)
            torch.cuda.synchronize()
            err = float((x - ref).abs().max() / ref.abs().max())
            assert err <= 1e-10, (prec, err)
        sols[prec] = x.clone()
        s.close()
    err = float((sols["mixed"] - sols["fp64"]).abs().max() / sols["fp64"].abs().max())
    assert err <= 1e-8, err
