"""bem_factor_rhs_planewave: compress_compact, factor and bem_rhs_planewave in one call, the
right-hand sides on a second stream beside the compression and the factor.  Every kernel
of the path is deterministic (fixed-order and exact fixed-point reductions), so the call
must reproduce the sequential calls bit for bit; a difference would be a race between the
two streams."""
import numpy as np
import pytest
import torch

from paper_2210_08580_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2210_08580_gb300 import bem
    bem.load_library()
    return bem


def _run(B, verts, k, ang, prec, memory, fused, alpha=0.0):
    s = B.Solver(device=0, prec=prec, memory=memory, refine_rtol=1e-8)
    s.assemble(torch.from_numpy(verts).cuda(), k, ops="SWD" if alpha else "SW")
    s.filter_apply(2 * 40 + 1, alpha=alpha)
    if fused:
        r, v = s.factor_rhs_planewave(1e-10, ang)
    else:
        r = s.compress(1e-10)
        s.factor()
        v = s.rhs_planewave(ang)
    x = s.solve(v)
    out = dict(r=r, v=v.clone(), x=x.clone(), sigma=s.matrix("sigma").clone(), U=s.matrix("U").clone(),
               Vh=s.matrix("Vh").clone())
    torch.cuda.synchronize()
    s.close()
    return out


@pytest.mark.parametrize("prec,memory", [("mixed", "torch"), ("mixed", "cuda"), ("fp64", "torch")])
def test_fused_call_reproduces_the_sequential_calls(B, prec, memory):
    verts, _, _ = I.equal_chord_mesh(I.random_star(3), 2048)
    ang = torch.from_numpy(I.planewave_angles(256))
    a = _run(B, verts, 2.0, ang, prec, memory, fused=False)
    b = _run(B, verts, 2.0, ang, prec, memory, fused=True)
    assert a["r"] == b["r"]
    for key in ("sigma", "U", "Vh", "v", "x"):
        assert torch.equal(a[key], b[key]), (key, float((a[key] - b[key]).abs().max()))


def test_fused_call_reproduces_the_sequential_calls_cfie(B):
    """the CFIE (alpha > 0): the right-hand sides add - alpha G^-1 h2 on the second stream"""
    verts, _, _ = I.equal_chord_mesh(I.random_star(4), 1024)
    ang = torch.from_numpy(I.planewave_angles(64))
    a = _run(B, verts, 3.0, ang, "mixed", "torch", fused=False, alpha=0.5)
    b = _run(B, verts, 3.0, ang, "mixed", "torch", fused=True, alpha=0.5)
    assert a["r"] == b["r"]
    for key in ("sigma", "U", "Vh", "v", "x"):
        assert torch.equal(a[key], b[key]), (key, float((a[key] - b[key]).abs().max()))


def test_fused_call_checks_its_arguments(B):
    verts, _, _ = I.equal_chord_mesh(I.cos_star(1.0, 0.3, 5), 301)
    s = B.Solver(device=0, prec="mixed")
    s.assemble(torch.from_numpy(verts).cuda(), 2.0, ops="SW")
    with pytest.raises(B.BemError):            # before filter_apply
        s.factor_rhs_planewave(1e-10, np.array([0.0]))
    s.filter_apply(41)
    r, v = s.factor_rhs_planewave(1e-10, np.array([0.0, 1.0]))
    assert r >= 1 and v.shape == (2, 301) and bool(torch.isfinite(v.real).all())
    s.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_fused_call_reproduces_the_sequential_calls_general_mesh(B, prec):
    """a non-equal-chord mesh: the right-hand sides' Gram solves (chunked, with their own
    scratch) run on the second stream beside the compression's"""
    verts, _ = I.parameter_mesh(I.random_star(5), 1500, grade=0.2)
    ang = torch.from_numpy(I.planewave_angles(128))
    a = _run(B, verts, 2.0, ang, prec, "torch", fused=False)
    b = _run(B, verts, 2.0, ang, prec, "torch", fused=True)
    assert a["r"] == b["r"]
    for key in ("sigma", "U", "Vh", "v", "x"):
        assert torch.equal(a[key], b[key]), (key, float((a[key] - b[key]).abs().max()))
