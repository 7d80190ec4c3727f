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


# ------------------------------------------------------------------ the C5 configuration
# Random Fourier star of seed 200 (16 coefficients), N = 8192, k = 1, n = 201 without
# truncation, 128 plane waves, 360 observation angles; target = the far field of the seed-201
# star.  The oracle's misfit, amplitude gradient and central differences in four
# coefficients are stored by tests/golden/make_goldens.py (run_c5).

import os

C5_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c5_fourier_star200_n8192.npz")


def _c5():
    with np.load(C5_PATH) as z:
        return {key: z[key] for key in z.files}


def _c5_J(B, g, coef, prec, grad=False):
    c = torch.tensor(coef, dtype=torch.float64, requires_grad=grad)
    a = torch.ones(128, dtype=torch.complex128, device="cuda", requires_grad=grad)
    obs = 2 * math.pi * np.arange(360) / 360
    u = B.shape_farfield(c, a, 1.0, int(g["N"]), float(g["k"]), 2 * int(g["M"]) + 1, I.planewave_angles(128), obs,
                         prec=prec)
    J = ((u - torch.from_numpy(g["target"].T.copy()).cuda()).abs() ** 2).sum()
    if grad:
        J.backward()
        return J.item(), c.grad.numpy(), a.grad.cpu().numpy()
    return J.item()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_c5_misfit_and_gradients_against_the_oracle(B, prec):
    """C5 on both paths: the misfit and its amplitude gradient against the oracle's, and the
    adjoint shape gradient against the oracle's central differences (h = 1e-6)."""
    g = _c5()
    J, gc, ga = _c5_J(B, g, g["coef"], prec, grad=True)
    tJ, ta = (1e-9, 1e-8) if prec == "fp64" else (1e-7, 1e-6)
    assert abs(J - float(g["J"])) <= tJ * float(g["J"]), (J, float(g["J"]))
    assert np.max(np.abs(ga - g["grad_a"])) <= ta * np.max(np.abs(g["grad_a"]))
    fd = g["fd"]
    for p, ref in zip(g["coefs_fd"], fd):
        assert abs(gc[p] - ref) <= 1e-5 * np.max(np.abs(fd)), (prec, int(p), gc[p], ref)
    print(f"C5 {prec}: J {J:.6e} (oracle {float(g['J']):.6e}), shape gradient at the differenced coefficients "
          f"{[float(gc[p]) for p in g['coefs_fd']]} vs {list(map(float, fd))}")


def test_c5_shape_gradient_matches_gpu_central_differences(B):
    g = _c5()
    _, gc, _ = _c5_J(B, g, g["coef"], "fp64", grad=True)
    h = float(g["h"])
    for p in g["coefs_fd"][:2]:
        e = np.zeros_like(g["coef"])
        e[p] = h
        fd = (_c5_J(B, g, g["coef"] + e, "fp64") - _c5_J(B, g, g["coef"] - e, "fp64")) / (2 * h)
        assert abs(fd - gc[p]) <= 1e-5 * np.max(np.abs(gc)), (int(p), fd, gc[p])
