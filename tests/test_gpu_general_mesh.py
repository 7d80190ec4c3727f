"""Non-equal-chord meshes on the GPU path (Sec. III-A: the orthonormalised Laplacian
L~ = G^-1/2 L G^-1/2 of non-homogeneous discretisations), against the oracle's literal
route (dense eigendecomposition of L~, dense SVD of P C2, Woodbury), element by element.

Meshes: polar-angle meshes of the perturbed circle r = 2 + 0.2 sin 8t, smoothly graded
(adjacent chords differ by up to about 1.6x across the curve) and uniform in the angle (the
Table I geometry, chords following the curve's speed), N = 300 (ten assembly tiles and a
ragged tail).  G and L are general cyclic tridiagonal there, G^-1 runs through the bordered
LDL^T factor and the filter basis through the shifted subspace iteration.
"""
import os

import numpy as np
import pytest
import torch

from oracle import bem_oracle as O
from paper_2210_08580_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ENTRY_TOL = 1e-13
SOLVE_TOL = 1e-10
MIXED_TOL = 1e-8
N_MODES = 21
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


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
def graded():
    v, _ = I.parameter_mesh(I.perturbed_circle(), 300, grade=0.25, phase=0.7)
    k = 1.3
    mats = O.assemble(v, k, "SWD")
    ang = I.planewave_angles(5)
    f = O.rhs_planewave(v, k, ang)
    h2 = O.rhs_planewave_h(v, k, ang)
    G = O.gram(v)
    vx = np.linalg.solve(G, mats["S"] @ np.linalg.solve(G, f))
    return dict(v=v, k=k, mats=mats, ang=ang, f=f, G=G, vx=vx,
                efie=O.filtered_solve_literal(mats, v, f, N_MODES, 1e-10),
                efie_t=O.filtered_solve_literal(mats, v, f, N_MODES, 1e-4),
                cfie=O.filtered_solve_literal(mats, v, f, N_MODES, 1e-10, alpha=0.5, h2=h2),
                nokernel=O.filtered_solve_literal(mats, v, f, N_MODES, 1e-10, include_kernel=False))


def _solver(B, c, ops="SW", **kw):
    s = B.Solver(device=0, **kw)
    s.assemble(_cuda(c["v"]), c["k"], ops=ops)
    return s


def test_general_mesh_is_detected_and_assembled(B, graded):
    c = graded
    s = _solver(B, c, "SWD")
    assert s.info()["equal_chord"] == 0
    for op in "SWD":
        assert _rel(_np(s.matrix(op)), c["mats"][op]) <= ENTRY_TOL, op
    s.close()


def test_general_gram_solves_in_the_rhs(B, graded):
    """v = G^-1 S G^-1 f with the general Gram matrix (bordered LDL^T solves)."""
    c = graded
    s = _solver(B, c)
    f, vv = s.rhs_planewave(_cuda(c["ang"]), want_f=True)
    assert _rel(_np(f).T, c["f"]) <= 1e-13
    assert _rel(_np(vv).T, c["vx"]) <= 1e-12, _rel(_np(vv).T, c["vx"])
    s.close()


@pytest.mark.parametrize("inc", [True, False])
def test_general_filter_basis_spans_the_lowest_eigenvectors(B, graded, inc):
    """Q is G-orthonormal and G^1/2 Q Q^T G^1/2 is the literal filter P^L_n (eigenvectors of
    L~, kernel mode kept or dropped)."""
    c = graded
    s = _solver(B, c, include_kernel_mode=inc)
    s.filter_apply(N_MODES)
    Q = _np(s.matrix("Q"))
    assert Q.shape == (300, N_MODES if inc else N_MODES - 1)
    G = c["G"]
    assert np.max(np.abs(Q.T @ G @ Q - np.eye(Q.shape[1]))) <= 1e-12
    P, _ = O.filter_literal(c["v"], N_MODES, include_kernel=inc)
    Gh = O._sym_pow(G, 0.5)
    assert np.max(np.abs(Gh @ Q @ Q.T @ Gh - P)) <= 1e-11
    s.close()


def test_general_filter_block_acts_as_the_literal_operator(B, graded):
    """Q B is the filtered compact part P_x C_x in nodal coordinates: G^1/2 (Q B) G^-1/2 equals
    the literal route's P C2 (B itself depends on the basis chosen inside span(Q))."""
    c = graded
    s = _solver(B, c)
    s.filter_apply(N_MODES)
    Q, Bg = _np(s.matrix("Q")), _np(s.matrix("B"))
    lit = c["efie"]
    PC = lit["Gh"] @ (Q @ Bg) @ lit["Gmh"]
    assert _rel(PC, lit["PC"]) <= 1e-11, _rel(PC, lit["PC"])
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_general_compression_and_solve_match_oracle(B, graded, prec):
    c = graded
    tol_x = SOLVE_TOL if prec == "fp64" else MIXED_TOL
    for key, tol in (("efie", 1e-10), ("efie_t", 1e-4)):
        ref = c[key]
        s = _solver(B, c, prec=prec)
        s.filter_apply(N_MODES)
        r = s.compress(tol)
        sig = _np(s.matrix("sigma"))
        assert np.max(np.abs(sig - ref["sigma"][:N_MODES])) <= 1e-11 * ref["sigma"][0]
        assert abs(r - ref["rank"]) <= 1
        s.factor()
        x = _np(s.solve(s.rhs_planewave(_cuda(c["ang"])))).T
        if r == ref["rank"]:
            assert _rel(x, ref["x"]) <= tol_x, (key, prec, _rel(x, ref["x"]))
        else:
            assert _rel(x, ref["x"]) <= 10 * tol
        s.close()


def test_general_cfie_and_literal_filter_match_oracle(B, graded):
    c = graded
    s = _solver(B, c, "SWD")
    s.filter_apply(N_MODES, alpha=0.5)
    assert s.compress(1e-10) == c["cfie"]["rank"]
    s.factor()
    x = _np(s.solve(s.rhs_planewave(_cuda(c["ang"])))).T
    assert _rel(x, c["cfie"]["x"]) <= SOLVE_TOL
    s.close()
    s = _solver(B, c, include_kernel_mode=False)
    s.filter_apply(N_MODES)
    assert s.compress(1e-10) == c["nokernel"]["rank"]
    s.factor()
    x = _np(s.solve(s.rhs_planewave(_cuda(c["ang"])))).T
    assert _rel(x, c["nokernel"]["x"]) <= SOLVE_TOL
    s.close()


def test_table1_geometry_uniform_in_angle(B):
    """The Table I curve meshed uniformly in the polar angle (chords follow the curve's speed,
    spread 1.4x), the paper's filtering point 200 (n = 201) on its smallest mesh N = 1004,
    line source at (3, 0),
    k = 0.4: solution, rank and singular values against the oracle's literal route."""
    v, _ = I.parameter_mesh(I.perturbed_circle(), 1004)
    k, n, tol = 0.4, 201, 1e-3
    mats = O.assemble(v, k, "SW")
    src = np.array([[3.0, 0.0]])
    f = O.rhs_pointsource(v, k, src)
    ref = O.filtered_solve_literal(mats, v, f, n, tol)
    s = B.Solver(device=0)
    s.assemble(_cuda(v), k, ops="SW")
    assert s.info()["equal_chord"] == 0
    vv = s.rhs_pointsource(_cuda(src))
    s.filter_apply(n)
    r = s.compress(tol)
    sig = _np(s.matrix("sigma"))
    assert np.max(np.abs(sig - ref["sigma"][:n])) <= 1e-11 * ref["sigma"][0]
    assert r == ref["rank"]
    s.factor()
    x = _np(s.solve(vv)).T
    assert _rel(x, ref["x"]) <= SOLVE_TOL, _rel(x, ref["x"])
    s.close()



@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_table1_n2008_against_stored_oracle(B, prec):
    """The Table I curve meshed uniformly in the polar angle at the paper's N = 2008, n = 201,
    tol 1e-3, k = 0.4: v, sigma, rank and the solutions for the line source at (3, 0) and four
    plane waves at 256 rows against the oracle's literal route, stored by
    tests/golden/make_goldens.py --only general."""
    g = np.load(os.path.join(GOLDEN, "general_table1_n2008.npz"))
    N, k, n, tol = int(g["N"]), float(g["k"]), int(g["n"]), float(g["tol"])
    v, _ = I.parameter_mesh(I.perturbed_circle(), N)
    s = B.Solver(device=0, prec=prec)
    s.assemble(_cuda(v), k, ops="SW")
    assert s.info()["equal_chord"] == 0
    vv = torch.cat([s.rhs_pointsource(_cuda(g["source"])), s.rhs_planewave(_cuda(g["angles"]))], dim=0)
    rows = g["rows"]
    v_tol = 1e-12 if prec == "fp64" else 5e-10
    assert _rel(_np(vv).T[rows], g["vx"]) <= v_tol, _rel(_np(vv).T[rows], g["vx"])
    s.filter_apply(n)
    r = s.compress(tol)
    sig = _np(s.matrix("sigma"))
    sig_tol = 1e-11 if prec == "fp64" else 1e-9
    assert np.max(np.abs(sig - g["sigma"])) <= sig_tol * g["sigma"][0]
    assert r == int(g["rank"])
    s.factor()
    x = _np(s.solve(vv)).T[rows]
    x_tol = SOLVE_TOL if prec == "fp64" else MIXED_TOL
    assert _rel(x, g["x"]) <= x_tol, (prec, _rel(x, g["x"]))
    s.close()


def test_general_farfield_and_adjoint_gradient(B, graded):
    """The far-field operator and the amplitude gradient of a far-field misfit on the graded
    mesh (the differentiation layer's entry points that do not differentiate the mesh):
    F x against the oracle's far-field matrix, and the gradient of J(a) = sum |F A^-1 (a_w v_w)
    - t|^2 through torch.autograd against the oracle's dense-LU gradient on the literal route's
    operator."""
    c = graded
    obs = np.linspace(0.0, 2 * np.pi, 24, endpoint=False)
    F = O.farfield_matrix(c["v"], c["k"], obs)
    s = _solver(B, c)
    s.filter_apply(N_MODES)
    s.compress(1e-10)
    s.factor()
    x = c["efie"]["x"]
    u = _np(s.farfield(_cuda(obs), _cuda(x.T))).T
    assert _rel(u, F @ x) <= 1e-12, _rel(u, F @ x)
    # misfit gradient in the amplitudes: A x = v with the literal route's operator in x
    # coordinates, A = beta I + G^-1/2 P C2 G^1/2
    lit = c["efie"]
    A = lit["Gmh"] @ (lit["beta"] * np.eye(len(c["v"])) + lit["U"] @ lit["Vh"]) @ lit["Gh"]
    a = np.array([1.0 + 0.5j, -0.3 + 0.2j, 0.7, 0.1j, -0.4])
    rng = np.random.default_rng(5)
    t = rng.standard_normal((len(obs), 5)) + 1j * rng.standard_normal((len(obs), 5))
    V = c["vx"]
    Xa = np.linalg.solve(A, V * a[None, :])
    R = F @ Xa - t
    J_ref = float(np.sum(np.abs(R) ** 2))
    # J through torch.autograd on the GPU path; its gradient (dJ/dRe a + i dJ/dIm a, the
    # binding's convention) against central differences of the oracle's J
    v0 = s.rhs_planewave(_cuda(c["ang"]))
    ag = _cuda(a).requires_grad_(True)
    uu = B.farfield_solve(ag[:, None] * v0, s, _cuda(obs))
    J = ((uu - _cuda(t.T)).abs() ** 2).sum()
    J.backward()
    assert abs(J.item() - J_ref) <= 1e-10 * J_ref, (J.item(), J_ref)
    def J_of(av):
        return float(np.sum(np.abs(F @ np.linalg.solve(A, V * av[None, :]) - t) ** 2))
    eps = 1e-6
    g = np.zeros(5, dtype=complex)
    for w in range(5):
        e = np.zeros(5); e[w] = eps
        dr = (J_of(a + e) - J_of(a - e)) / (2 * eps)
        di = (J_of(a + 1j * e) - J_of(a - 1j * e)) / (2 * eps)
        g[w] = dr + 1j * di
    assert _rel(ag.grad.cpu().numpy(), g) <= 1e-6, (ag.grad.cpu().numpy(), g)
    s.close()


@pytest.mark.parametrize("N,n", [(16, 7), (40, 31), (65, 9)])
def test_general_mesh_edge_sizes(B, N, n):
    """Edge cases of the general-mesh kernels against the literal route: the smallest mesh (one
    chunk in the chunked factor and solves), a filter whose subspace block is capped at N - 1
    (n = 31 of N = 40), and a chunk boundary one past a multiple of 64."""
    v, _ = I.parameter_mesh(I.cos_star(1.0, 0.3, 5), N, grade=0.3)
    k = 1.0
    mats = O.assemble(v, k, "SW")
    ang = I.planewave_angles(3)
    f = O.rhs_planewave(v, k, ang)
    ref = O.filtered_solve_literal(mats, v, f, n, 1e-12)
    s = B.Solver(device=0)
    s.assemble(_cuda(v), k, ops="SW")
    assert s.info()["equal_chord"] == 0
    vv = s.rhs_planewave(_cuda(ang))
    G = O.gram(v)
    vx = np.linalg.solve(G, mats["S"] @ np.linalg.solve(G, f))
    assert _rel(_np(vv).T, vx) <= 1e-12
    s.filter_apply(n)
    assert s.info()["basis_block"] == min(n + n // 2 + 9, N - 1)
    r = s.compress(1e-12)
    assert abs(r - ref["rank"]) <= 1
    s.factor()
    x = _np(s.solve(vv)).T
    if r == ref["rank"]:
        assert _rel(x, ref["x"]) <= SOLVE_TOL, _rel(x, ref["x"])
    s.close()
