"""Seeded synthetic inputs: closed star-shaped curves, their equal-chord P1 meshes
and plane-wave incidence angles.

This module holds none of the solver's arithmetic. It produces the vertex arrays
that both the CUDA path and the CPU oracle read, so that the two sides always see
identical geometry.

Curves (the paper evaluates on an ellipse and on a perturbed circle, Sec. V; the
other shapes are the synthetic workloads of this project):

* ``circle(a)``                      r(theta) = a
* ``cos_star(r0, amp, m)``           r(theta) = r0 + amp cos(m theta)
* ``random_star(seed)``              r(theta) = 1 + sum_{m=1..8} a_m cos(m theta + phi_m),
                                     a_m = 0.15/m * U[0,1), phi_m = 2 pi U[0,1), drawn
                                     in the order (a_1, phi_1, ..., a_8, phi_8) from
                                     ``numpy.random.default_rng(seed)``
* ``fourier_star(alpha, beta)``      r(theta) = 1 + sum_m alpha_m cos(m theta) + beta_m sin(m theta)
* ``perturbed_circle()``             r(theta) = 2 + 0.2 sin(8 theta)   (Sec. V, Table I)
* ``ellipse(a, b)``                  polar form of the ellipse with semi-axes a, b (Sec. V)

Meshes are *equal-chord* by default: vertices r_i = r(theta_i) (cos theta_i, sin theta_i),
theta_0 = 0, counter-clockwise, with |r_{i+1} - r_i| = h for every i including the
closing chord.  The paper does not say how its meshes are built; equal chords make
the P1 Gram and Laplacian matrices exactly circulant, which is the setting in which
the Laplacian filter can be applied with Fourier modes (Sec. III-A).  ``parameter_mesh``
builds the non-equal-chord meshes (uniform or smoothly graded in the polar angle), for
which the paper's orthonormalised Laplacian has no closed-form eigenvectors.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "PolarCurve", "circle", "cos_star", "random_star", "fourier_star",
    "perturbed_circle", "ellipse", "equal_chord_mesh", "regular_polygon",
    "planewave_angles", "batch_problems", "BatchProblem", "equal_chord_tangent",
    "parameter_mesh",
]


@dataclasses.dataclass(frozen=True)
class PolarCurve:
    """r(theta) = r0 + sum_m (cos_coef[m-1] cos(m theta) + sin_coef[m-1] sin(m theta)).

    ``ellipse_ab`` switches to the polar form of an ellipse instead.
    """
    r0: float = 1.0
    cos_coef: tuple = ()
    sin_coef: tuple = ()
    ellipse_ab: tuple | None = None
    name: str = "curve"

    def radius(self, th):
        th = np.asarray(th, dtype=np.float64)
        if self.ellipse_ab is not None:
            a, b = self.ellipse_ab
            return a * b / np.sqrt((b * np.cos(th)) ** 2 + (a * np.sin(th)) ** 2)
        r = np.full_like(th, self.r0)
        for m, c in enumerate(self.cos_coef, start=1):
            r = r + c * np.cos(m * th)
        for m, s in enumerate(self.sin_coef, start=1):
            r = r + s * np.sin(m * th)
        return r

    def dradius(self, th):
        th = np.asarray(th, dtype=np.float64)
        if self.ellipse_ab is not None:
            a, b = self.ellipse_ab
            den = (b * np.cos(th)) ** 2 + (a * np.sin(th)) ** 2
            dden = 2.0 * (a * a - b * b) * np.sin(th) * np.cos(th)
            return -0.5 * a * b * dden / den ** 1.5
        d = np.zeros_like(th)
        for m, c in enumerate(self.cos_coef, start=1):
            d = d - m * c * np.sin(m * th)
        for m, s in enumerate(self.sin_coef, start=1):
            d = d + m * s * np.cos(m * th)
        return d

    def point(self, th):
        r = self.radius(th)
        return np.stack([r * np.cos(th), r * np.sin(th)], axis=-1)

    def dpoint(self, th):
        r = self.radius(th)
        dr = self.dradius(th)
        c, s = np.cos(th), np.sin(th)
        return np.stack([dr * c - r * s, dr * s + r * c], axis=-1)


def circle(a: float = 1.0) -> PolarCurve:
    return PolarCurve(r0=float(a), name=f"circle(a={a})")


def cos_star(r0: float = 1.0, amp: float = 0.3, m: int = 5) -> PolarCurve:
    cos_coef = [0.0] * m
    cos_coef[m - 1] = float(amp)
    return PolarCurve(r0=float(r0), cos_coef=tuple(cos_coef), name=f"star({r0}+{amp}cos{m}t)")


def random_star(seed: int, harmonics: int = 8, amp: float = 0.15) -> PolarCurve:
    """r = 1 + sum a_m cos(m theta + phi_m), a_m = amp/m U, phi_m = 2 pi U (seeded)."""
    rng = np.random.default_rng(seed)
    u = rng.random(2 * harmonics)
    a = np.array([amp / m * u[2 * (m - 1)] for m in range(1, harmonics + 1)])
    ph = np.array([2.0 * math.pi * u[2 * (m - 1) + 1] for m in range(1, harmonics + 1)])
    # a cos(m t + ph) = a cos(ph) cos(m t) - a sin(ph) sin(m t)
    return PolarCurve(r0=1.0, cos_coef=tuple(a * np.cos(ph)), sin_coef=tuple(-a * np.sin(ph)),
                      name=f"random_star(seed={seed})")


def fourier_star(alpha, beta) -> PolarCurve:
    return PolarCurve(r0=1.0, cos_coef=tuple(float(x) for x in alpha),
                      sin_coef=tuple(float(x) for x in beta), name="fourier_star")


def fourier_star_seeded(seed: int, harmonics: int = 8, amp: float = 0.15):
    """16 shape coefficients (alpha_m, beta_m) with |.| ~ amp/m U[-1,1) (seeded)."""
    rng = np.random.default_rng(seed)
    u = rng.random(2 * harmonics) * 2.0 - 1.0
    alpha = np.array([amp / m * u[2 * (m - 1)] for m in range(1, harmonics + 1)])
    beta = np.array([amp / m * u[2 * (m - 1) + 1] for m in range(1, harmonics + 1)])
    return alpha, beta


def perturbed_circle() -> PolarCurve:
    s = [0.0] * 8
    s[7] = 0.2
    return PolarCurve(r0=2.0, sin_coef=tuple(s), name="perturbed_circle(2+0.2sin8t)")


def ellipse(a: float = 1.42, b: float = 1.32) -> PolarCurve:
    return PolarCurve(ellipse_ab=(float(a), float(b)), name=f"ellipse({a},{b})")


def regular_polygon(N: int, a: float = 1.0) -> np.ndarray:
    """Vertices a (cos 2 pi i/N, sin 2 pi i/N): the equal-chord mesh of a circle."""
    th = 2.0 * math.pi * np.arange(N) / N
    return np.ascontiguousarray(np.stack([a * np.cos(th), a * np.sin(th)], axis=-1))


def parameter_mesh(curve: PolarCurve, N: int, grade: float = 0.0, phase: float = 0.0):
    """Vertices at theta_i = t_i + grade sin(t_i - phase), t_i = 2 pi i / N: returns
    (verts (N,2) f64, theta (N,)).  With grade = 0 the vertices are uniform in the polar
    angle (the chords then follow the curve's speed); 0 < |grade| < 1 grades them smoothly,
    adjacent chords of a circle differing by up to a factor (1 + |grade|)/(1 - |grade|)
    across the curve.  These are the non-equal-chord meshes, for which G and L are general
    cyclic tridiagonal matrices (Sec. III-A's orthonormalised Laplacian)."""
    if not abs(grade) < 1.0:
        raise ValueError("grade must lie in (-1, 1)")
    t = 2.0 * math.pi * np.arange(N) / N
    th = t + grade * np.sin(t - phase)
    return np.ascontiguousarray(curve.point(th)), th


def _arclength_thetas(curve: PolarCurve, N: int, fine: int | None = None) -> np.ndarray:
    """theta_i at equal arclength spacing (initial guess for the equal-chord solve)."""
    M = fine or max(64 * N, 8192)
    th = 2.0 * math.pi * np.arange(M) / M
    speed = np.linalg.norm(curve.dpoint(th), axis=-1)
    # periodic trapezoid rule: cumulative arclength at the fine nodes
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (speed + np.roll(speed, -1)))]) * (2.0 * math.pi / M)
    Ltot = cum[-1]
    th_f = np.concatenate([th, [2.0 * math.pi]])
    target = Ltot * np.arange(N) / N
    guess = np.interp(target, cum, th_f)
    # Newton polish on s(theta) = target using the speed as derivative (fine cumulative
    # integral re-evaluated by interpolation is accurate enough for a starting guess)
    return guess


def equal_chord_mesh(curve: PolarCurve, N: int, tol: float = 1e-15, max_iter: int = 30):
    """Equal-chord vertices of ``curve``: returns (verts (N,2) f64, theta (N,), h).

    The chords agree to within the rounding of the vertex coordinates (about
    1e-16 |r| / h relative).  Unknowns theta_1..theta_{N-1} and h; equations |P(theta_{i+1}) - P(theta_i)| = h for
    i = 0..N-1 with theta_0 = 0, theta_N = 2 pi.  Solved by Newton's method on the
    sparse (cyclic bidiagonal + one column) Jacobian, starting from arclength spacing.
    """
    from scipy.sparse import csc_matrix
    from scipy.sparse.linalg import spsolve

    th = _arclength_thetas(curve, N)
    th[0] = 0.0
    P = curve.point(th)
    h = float(np.mean(np.linalg.norm(np.roll(P, -1, axis=0) - P, axis=-1)))
    idx = np.arange(N)
    prev_err = np.inf
    for it in range(max_iter):
        th_ext = np.concatenate([th, [2.0 * math.pi]])
        P = curve.point(th_ext)
        dP = curve.dpoint(th_ext)
        d = P[1:] - P[:-1]                         # chord vectors, (N,2)
        c = np.linalg.norm(d, axis=-1)
        F = c - h
        err = float(np.max(np.abs(F)))
        # stop at tol, or once rounding of the vertex coordinates stalls the iteration
        if err <= tol * h or (it > 2 and err > 0.5 * prev_err):
            break
        prev_err = err
        u = d / c[:, None]
        # dF_i/dtheta_i = -u_i . P'(theta_i) ; dF_i/dtheta_{i+1} = u_i . P'(theta_{i+1})
        a_diag = -np.einsum("ij,ij->i", u, dP[:-1])
        a_sup = np.einsum("ij,ij->i", u, dP[1:])
        rows, cols, vals = [], [], []
        # column j of the unknown vector: j = 0..N-2 -> theta_{j+1}; j = N-1 -> h
        for_i = idx[1:]                             # theta_i is unknown for i >= 1
        rows.append(for_i); cols.append(for_i - 1); vals.append(a_diag[1:])
        sup_i = idx[:-1]                            # theta_{i+1} unknown for i+1 <= N-1
        rows.append(sup_i); cols.append(sup_i); vals.append(a_sup[:-1])
        rows.append(idx); cols.append(np.full(N, N - 1)); vals.append(-np.ones(N))
        J = csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(N, N))
        delta = spsolve(J, -F)
        th = th.copy()
        th[1:] += delta[:-1]
        h += float(delta[-1])
    verts = np.ascontiguousarray(curve.point(th))
    return verts, th, h


def equal_chord_tangent(curve: PolarCurve, theta, h: float) -> np.ndarray:
    """Derivatives of the equal-chord vertices with respect to the curve's Fourier
    coefficients p = (cos_coef..., sin_coef...): returns (P, N, 2).

    The mesh solves F_i = |P(theta_{i+1}) - P(theta_i)| - h = 0 (theta_0 = 0, theta_N = 2 pi)
    for theta_1..theta_{N-1} and h; differentiating at fixed p gives
    J d(theta, h)/dp = -dF/dp with the Newton Jacobian J of ``equal_chord_mesh``, and
    d r_i/dp = P'(theta_i) d theta_i/dp + dP/dp(theta_i), dP/dp(theta) = basis(theta) (cos, sin)."""
    from scipy.sparse import csc_matrix
    from scipy.sparse.linalg import splu

    th = np.asarray(theta, dtype=np.float64)
    N = th.shape[0]
    th_ext = np.concatenate([th, [2.0 * math.pi]])
    P = curve.point(th_ext)
    dP = curve.dpoint(th_ext)
    d = P[1:] - P[:-1]
    u = d / np.linalg.norm(d, axis=-1)[:, None]
    idx = np.arange(N)
    a_diag = -np.einsum("ij,ij->i", u, dP[:-1])
    a_sup = np.einsum("ij,ij->i", u, dP[1:])
    rows = np.concatenate([idx[1:], idx[:-1], idx])
    cols = np.concatenate([idx[1:] - 1, idx[:-1], np.full(N, N - 1)])
    vals = np.concatenate([a_diag[1:], a_sup[:-1], -np.ones(N)])
    lu = splu(csc_matrix((vals, (rows, cols)), shape=(N, N)))
    mc, ms = len(curve.cos_coef), len(curve.sin_coef)
    basis = [(lambda t, m=m: np.cos(m * t)) for m in range(1, mc + 1)] + \
            [(lambda t, m=m: np.sin(m * t)) for m in range(1, ms + 1)]
    out = np.zeros((len(basis), N, 2))
    dir_ext = np.stack([np.cos(th_ext), np.sin(th_ext)], axis=-1)
    for p_, b in enumerate(basis):
        dPp = b(th_ext)[:, None] * dir_ext                      # dP/dp at the nodes
        dF = np.einsum("ij,ij->i", u, dPp[1:] - dPp[:-1])
        sol = lu.solve(-dF)
        dth = np.concatenate([[0.0], sol[:-1]])
        out[p_] = dP[:-1] * dth[:, None] + dPp[:-1]
    return out


def planewave_angles(nrhs: int) -> np.ndarray:
    """Incidence angles phi_w = 2 pi w / nrhs, w = 0..nrhs-1."""
    return 2.0 * math.pi * np.arange(nrhs, dtype=np.float64) / nrhs


@dataclasses.dataclass(frozen=True)
class BatchProblem:
    seed: int
    curve: PolarCurve
    N: int
    k: float
    nrhs: int


def batch_problems(count: int = 64, first_seed: int = 100, n_lo: int = 512, n_hi: int = 8192,
                   k_lo: float = 1e-2, k_hi: float = 5.0, r_lo: int = 64, r_hi: int = 512):
    """Uneven many-geometry batch: per problem i, ``default_rng(first_seed + i)`` draws
    the 16 shape numbers of ``random_star`` first, then N ~ U{n_lo..n_hi},
    k = 10^U(log10 k_lo, log10 k_hi), nrhs ~ U{r_lo..r_hi}."""
    out = []
    for i in range(count):
        seed = first_seed + i
        rng = np.random.default_rng(seed)
        rng.random(16)
        N = int(rng.integers(n_lo, n_hi + 1))
        k = float(10.0 ** rng.uniform(math.log10(k_lo), math.log10(k_hi)))
        nrhs = int(rng.integers(r_lo, r_hi + 1))
        out.append(BatchProblem(seed=seed, curve=random_star(seed), N=N, k=k, nrhs=nrhs))
    return out
