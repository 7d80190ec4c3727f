"""The seeded input generators: equal-chord meshes and their derivative in the curve's
Fourier coefficients (central differences of the mesh generator itself)."""
import numpy as np

from paper_2210_08580_gb300 import inputs as I


def test_equal_chord_mesh_has_equal_chords():
    v, th, h = I.equal_chord_mesh(I.random_star(3), 200)
    chords = np.linalg.norm(np.roll(v, -1, axis=0) - v, axis=1)
    assert np.max(np.abs(chords - h)) <= 1e-13 * h
    assert th[0] == 0.0 and np.all(np.diff(th) > 0)


def test_equal_chord_tangent_matches_central_differences():
    al, be = np.array([0.05, 0.02, -0.01]), np.array([0.03, -0.01, 0.015])
    N = 80
    c = I.fourier_star(al, be)
    v, th, h = I.equal_chord_mesh(c, N)
    T = I.equal_chord_tangent(c, th, h)
    eps = 1e-6
    for p in range(6):
        dp = np.zeros(6)
        dp[p] = eps
        vp, _, _ = I.equal_chord_mesh(I.fourier_star(al + dp[:3], be + dp[3:]), N)
        vm, _, _ = I.equal_chord_mesh(I.fourier_star(al - dp[:3], be - dp[3:]), N)
        fd = (vp - vm) / (2 * eps)
        assert np.max(np.abs(fd - T[p])) <= 1e-8 * max(1.0, np.max(np.abs(T[p])))
