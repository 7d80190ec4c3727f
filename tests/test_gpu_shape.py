"""Shape gradient of a far-field misfit (bem_shape_vjp behind torch.autograd): against
central differences of the GPU misfit and of the CPU oracle's misfit in the curve's Fourier
coefficients (each difference rebuilds the equal-chord mesh), and the amplitude gradient
against the oracle's adjoint formula."""
import math

import numpy as np
import pytest
import torch

from oracle import bem_oracle as O
from paper_2210_08580_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N, K, M = 96, 1.3, 10
COEF = np.array([0.06, -0.03, 0.04, 0.02])          # cos_1, cos_2, sin_1, sin_2
ANG = np.array([0.0, 2.1, 4.2])
OBS = np.linspace(0.0, 2 * math.pi, 12, endpoint=False)
AMP = np.array([1.0 + 0.2j, 0.6 - 0.3j, -0.5 + 0.4j])
H = 1e-6


@pytest.fixture(scope="module")
def B():
    from paper_2210_08580_gb300 import bem
    bem.load_library()
    return bem


@pytest.fixture(scope="module")
def target():
    rng = np.random.default_rng(5)
    return 0.05 * (rng.standard_normal((3, 12)) + 1j * rng.standard_normal((3, 12)))


def _gpu_J(B, coef, amp, target, grad=False):
    c = torch.tensor(coef, dtype=torch.float64, requires_grad=grad)
    a = torch.tensor(amp, dtype=torch.complex128, device="cuda", requires_grad=grad)
    u = B.shape_farfield(c, a, 1.0, N, K, 2 * M + 1, ANG, OBS)
    J = ((u - torch.from_numpy(target).cuda()).abs() ** 2).sum()
    if grad:
        J.backward()
        return J.item(), c.grad.numpy(), a.grad.cpu().numpy()
    return J.item()


def _oracle_J(coef, amp, target):
    m = len(coef) // 2
    curve = I.PolarCurve(r0=1.0, cos_coef=tuple(coef[:m]), sin_coef=tuple(coef[m:]))
    v, _, _ = I.equal_chord_mesh(curve, N)
    mats = O.assemble(v, K, "SW")
    route = O.filtered_solve_projected(mats, v, O.rhs_planewave(v, K, ANG), M, 0.0)
    return O.misfit_and_gradients(route, O.farfield_matrix(v, K, OBS), amp, target.T)


def test_shape_gradient_matches_gpu_central_differences(B, target):
    J, gc, _ = _gpu_J(B, COEF, AMP, target, grad=True)
    for p in range(len(COEF)):
        e = np.zeros_like(COEF)
        e[p] = H
        fd = (_gpu_J(B, COEF + e, AMP, target) - _gpu_J(B, COEF - e, AMP, target)) / (2 * H)
        assert abs(fd - gc[p]) <= 1e-5 * max(np.max(np.abs(gc)), 1e-12), (p, fd, gc[p])


def test_shape_and_amplitude_gradients_match_the_oracle(B, target):
    J, gc, ga = _gpu_J(B, COEF, AMP, target, grad=True)
    ref = _oracle_J(COEF, AMP, target)
    assert abs(J - ref["J"]) <= 1e-9 * ref["J"]
    assert np.max(np.abs(ga - ref["grad_a"])) <= 1e-8 * np.max(np.abs(ref["grad_a"]))
    for p in range(len(COEF)):
        e = np.zeros_like(COEF)
        e[p] = H
        fd = (_oracle_J(COEF + e, AMP, target)["J"] - _oracle_J(COEF - e, AMP, target)["J"]) / (2 * H)
        assert abs(fd - gc[p]) <= 1e-5 * max(np.max(np.abs(gc)), 1e-12), (p, fd, gc[p])
