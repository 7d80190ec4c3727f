"""One handle driven through problems of changing size gives the same bits as fresh handles.

A handle keeps its stage buffers from call to call (they grow when a later call needs more
and are freed when N changes), and every kernel on the path is deterministic (fixed-point
cross-CTA sums in the QR, integer exponent maxima, fixed reduction orders), so reuse must
not change a single bit of the solution."""
import pytest
import torch

from paper_2210_08580_gb300 import inputs as I

pytestmark = pytest.mark.gpu

K = 2.0
ANG = I.planewave_angles(5)


@pytest.fixture(scope="module")
def B():
    from paper_2210_08580_gb300 import bem
    bem.load_library()
    return bem


def _meshes():
    star = I.cos_star(1.0, 0.3, 5)
    return {N: torch.from_numpy(I.equal_chord_mesh(star, N)[0]) for N in (200, 256)}


def _run(s, verts, n_modes, tol=1e-10):
    s.assemble(verts, K, ops="SW")
    s.filter_apply(n_modes)
    r = s.compress(tol)
    s.factor()
    v = s.rhs_planewave(ANG)
    return s.solve(v).cpu(), r


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_reused_handle_matches_fresh_handles(B, prec):
    meshes = _meshes()
    # sequence: more modes (the filter and compression buffers grow), fewer again (reused
    # larger buffers), then a new N (everything freed and reallocated), then the first case
    seq = [(200, 21), (200, 41), (200, 21), (256, 31), (200, 21)]
    reused = B.Solver(device=0, prec=prec)
    got = [_run(reused, meshes[N], n) for N, n in seq]
    reused.close()
    for (N, n), (x, r) in zip(seq, got):
        fresh = B.Solver(device=0, prec=prec)
        x0, r0 = _run(fresh, meshes[N], n)
        fresh.close()
        assert r == r0, (N, n)
        assert torch.equal(x, x0), (N, n, float((x - x0).abs().max()))
    # and the two visits of the first case agree with each other
    assert torch.equal(got[0][0], got[2][0]) and torch.equal(got[0][0], got[4][0])


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_handle_between_equal_chord_and_general_meshes(B, prec):
    """The same N meshed with equal chords and at graded polar angles, alternately, on one
    handle: the general mesh's factor, basis and G Q must not leak into the equal-chord
    problem (nor the other way round)."""
    star = I.cos_star(1.0, 0.3, 5)
    eq = torch.from_numpy(I.equal_chord_mesh(star, 256)[0])
    gr = torch.from_numpy(I.parameter_mesh(star, 256, grade=0.3)[0])
    seq = [(eq, 21), (gr, 21), (eq, 21), (gr, 31), (gr, 21)]
    reused = B.Solver(device=0, prec=prec)
    got = []
    for v, n in seq:
        got.append(_run(reused, v, n))
        assert reused.info()["equal_chord"] == (1 if v is eq else 0)
    reused.close()
    for (v, n), (x, r) in zip(seq, got):
        fresh = B.Solver(device=0, prec=prec)
        x0, r0 = _run(fresh, v, n)
        fresh.close()
        assert r == r0
        assert torch.equal(x, x0), float((x - x0).abs().max())
