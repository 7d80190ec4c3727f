"""Differentiation layer on the GPU: the far-field operator and the adjoint gradient of a
far-field misfit (bem_farfield, bem_farfield_adjoint, solve_backward behind
torch.autograd), against the CPU oracle's far field and gradients and against central
differences of the misfit computed on the GPU."""
import numpy as np
import pytest
import torch

from oracle import bem_oracle as O
from paper_2210_08580_gb300 import inputs as I

pytestmark = pytest.mark.gpu

M = 20                      # n = 41 filter modes
TOL = 1e-10
K = 1.7


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def B():
    from paper_2210_08580_gb300 import bem
    bem.load_library()
    return bem


@pytest.fixture(scope="module")
def case():
    v, _, _ = I.equal_chord_mesh(I.cos_star(1.0, 0.3, 5), 301)
    ang = I.planewave_angles(4)
    mats = O.assemble(v, K, "SW")
    f = O.rhs_planewave(v, K, ang)
    route = O.filtered_solve_projected(mats, v, f, M, TOL)
    obs = np.linspace(0.0, 2 * np.pi, 36, endpoint=False)
    rng = np.random.default_rng(11)
    target = 0.02 * (rng.standard_normal((36, 4)) + 1j * rng.standard_normal((36, 4)))
    a = np.array([1.0 + 0.3j, 0.5 - 0.2j, -0.7 + 0.1j, 0.2 + 0.9j])
    return dict(v=v, ang=ang, route=route, obs=obs, F=O.farfield_matrix(v, K, obs), target=target, a=a,
                ref=O.misfit_and_gradients(route, O.farfield_matrix(v, K, obs), a, target))


def _solver(B, case, prec):
    s = B.Solver(device=0, prec=prec)
    s.assemble(_cuda(case["v"]), K, ops="SW")
    s.filter_apply(2 * M + 1)
    s.compress(TOL)
    s.factor()
    return s


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_farfield_and_adjoint_match_oracle(B, case):
    s = _solver(B, case, "fp64")
    x = case["ref"]["x0"]
    xg = _cuda(x.T)
    u = s.farfield(_cuda(case["obs"]), xg).cpu().numpy().T
    assert _rel(u, case["F"] @ x) <= 1e-12
    g = case["target"]
    adj = s.farfield_adjoint(_cuda(case["obs"]), _cuda(g.T)).cpu().numpy().T
    assert _rel(adj, case["F"].conj().T @ g) <= 1e-12
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_gradient_matches_oracle(B, case, prec):
    """grad of J(a) = sum |F A^-1 (a_w v_w) - t|^2 through torch.autograd (the backward is
    bem_farfield_adjoint + solve_backward) against the oracle's dense-LU gradient."""
    s = _solver(B, case, prec)
    v0 = s.rhs_planewave(_cuda(case["ang"]))
    a = _cuda(case["a"]).requires_grad_(True)
    u = B.farfield_solve(a[:, None] * v0, s, _cuda(case["obs"]))
    J = ((u - _cuda(case["target"].T)).abs() ** 2).sum()
    J.backward()
    ref = case["ref"]
    tol = 1e-10 if prec == "fp64" else 1e-8
    assert abs(J.item() - ref["J"]) <= tol * ref["J"]
    assert _rel(a.grad.cpu().numpy(), ref["grad_a"]) <= tol
    s.close()


def test_gradient_matches_central_differences(B, case):
    """Central differences (h = 1e-6) of the GPU misfit in each amplitude, real and
    imaginary directions, against the adjoint gradient."""
    s = _solver(B, case, "fp64")
    v0 = s.rhs_planewave(_cuda(case["ang"]))
    obs = _cuda(case["obs"])
    t = _cuda(case["target"].T)

    def J_of(a):
        with torch.no_grad():
            u = B.farfield_solve(a[:, None] * v0, s, obs)
            return ((u - t).abs() ** 2).sum().item()

    a = _cuda(case["a"]).requires_grad_(True)
    u = B.farfield_solve(a[:, None] * v0, s, obs)
    ((u - t).abs() ** 2).sum().backward()
    g = a.grad.detach().clone()
    h = 1e-6
    for w in range(4):
        for unit, part in ((1.0, g[w].real.item()), (1j, g[w].imag.item())):
            e = torch.zeros(4, dtype=torch.complex128, device="cuda")
            e[w] = h * unit
            fd = (J_of(a.detach() + e) - J_of(a.detach() - e)) / (2 * h)
            assert abs(fd - part) <= 1e-6 * max(1.0, abs(part)), (w, unit, fd, part)
    s.close()
