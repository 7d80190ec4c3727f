"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
continuous spectra on the circle (Graf's addition theorem), the exact Mie current,
an independent high-precision integrator (mpmath), the divergence theorem, the
Woodbury identity, printed values of Table I, and brute-force dense solves.
"""
import math
import os

import numpy as np
import pytest

from oracle import bem_oracle as O
from paper_2210_08580_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def circle_mats():
    out = {}
    for N in (64, 128):
        v = I.regular_polygon(N)
        out[N] = (v, O.assemble(v, 1.0, "SWD"))
    return out


@pytest.fixture(scope="module")
def star_case():
    v, _, _ = I.equal_chord_mesh(I.cos_star(1.0, 0.3, 5), 96)
    k = 1.3
    mats = O.assemble(v, k, "SWD")
    return v, k, mats


# ------------------------------------------------------------------ special functions


def test_bessel_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    from scipy import special
    zs = [1e-6, 1e-3, 0.05, 0.7, 2.0, 4.9, 7.99, 8.01, 12.5, 17.0, 26.0]
    for z in zs:
        for fn, ref in ((special.j0, lambda x: mp.besselj(0, x)), (special.y0, lambda x: mp.bessely(0, x)),
                        (special.j1, lambda x: mp.besselj(1, x)), (special.y1, lambda x: mp.bessely(1, x))):
            a = fn(z)
            b = float(ref(mp.mpf(z)))
            assert abs(a - b) <= 2e-15 * max(1.0, abs(b)), (fn, z, a, b)


def test_green_log_limit():
    # DLMF 10.8.2: g2(r) + ln(r)/(2 pi) -> i/4 - (ln(k/2) + gamma)/(2 pi) as r -> 0
    for k in (1e-3, 1.0, 5.0):
        r = 1e-9
        lim = 0.25j - (math.log(k / 2) + np.euler_gamma) / (2 * math.pi)
        val = O.green(k, r) + math.log(r) / (2 * math.pi)
        assert abs(val - lim) < 1e-12


# ------------------------------------------------------------------ quadrature


def _mp_pair(mp, k, x0, tx, hx, y0, ty, hy, a, b, split_inner_at_s=False, kernel="S", nu=None,
             method="tanh-sinh"):
    lam = lambda c, u, hh: (1 - u / hh) if c == 0 else (u / hh)

    def g(r):
        return 0.25j * mp.besselj(0, k * r) - 0.25 * mp.bessely(0, k * r)

    def dg(r, dn):
        return (-0.25j * k) * (mp.besselj(1, k * r) + 1j * mp.bessely(1, k * r)) / r * dn

    def inner(s):
        xs = (x0[0] + s * tx[0], x0[1] + s * tx[1])

        def f(t):
            yt = (y0[0] + t * ty[0], y0[1] + t * ty[1])
            dx, dy = yt[0] - xs[0], yt[1] - xs[1]
            r = mp.sqrt(dx * dx + dy * dy)
            ker = g(r) if kernel == "S" else dg(r, dx * nu[0] + dy * nu[1])
            return lam(a, s, hx) * lam(b, t, hy) * ker
        pts = [0, s, hy] if split_inner_at_s else [0, hy]
        return mp.quad(f, pts, method=method)
    return complex(mp.quad(inner, [0, hx], method=method))


@pytest.mark.parametrize("which", ["self", "adjacent", "near"])
def test_pair_integrals_against_mpmath(which):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 17
    v, _, _ = I.equal_chord_mesh(I.cos_star(1.0, 0.3, 5), 24)
    mesh = O.Mesh(v)
    k = 2.0
    e = 3
    f = {"self": 3, "adjacent": 4, "near": 6}[which]
    Iq, Jq, _ = O.pair_integrals(mesh, k, [e], [f], need_d=True)
    method = "gauss-legendre" if which == "near" else "tanh-sinh"
    for (a, b) in ((0, 1), (1, 1)):
        ref = _mp_pair(mp, k, mesh.P0[e], mesh.t[e], mesh.h[e], mesh.P0[f], mesh.t[f], mesh.h[f],
                       a, b, split_inner_at_s=(which == "self"), method=method)
        assert abs(Iq[0, a, b] - ref) <= 1e-13 * abs(ref), (which, a, b, Iq[0, a, b], ref)
        if which != "self" and (a, b) == (0, 1):
            refd = _mp_pair(mp, k, mesh.P0[e], mesh.t[e], mesh.h[e], mesh.P0[f], mesh.t[f], mesh.h[f],
                            a, b, kernel="D", nu=mesh.nu[f], method=method)
            assert abs(Jq[0, a, b] - refd) <= 1e-12 * abs(refd) + 1e-16, (which, a, b, Jq[0, a, b], refd)
    if which == "self":
        assert np.all(Jq == 0)


# ------------------------------------------------------------------ discrete operators


def test_circulant_and_symmetric(circle_mats):
    for N, (v, m) in circle_mats.items():
        for op in "SWD":
            A = m[op]
            shifted = np.roll(np.roll(A, 1, 0), 1, 1)
            assert np.max(np.abs(A - shifted)) <= 1e-13 * np.max(np.abs(A)), op
        for op in "SW":
            A = m[op]
            assert np.max(np.abs(A - A.T)) <= 1e-14 * np.max(np.abs(A)), op


def test_circle_spectra_second_order(circle_mats):
    """Eigenvalues of G^-1 X on the regular polygon converge at O(h^2) to the continuous
    circle spectra of S, N and D (sign and scale of all three operators)."""
    k = 1.0
    ms = np.arange(0, 3)
    errs = {}
    for N, (v, m) in circle_mats.items():
        G = O.gram(v).astype(complex)
        g = np.fft.fft(G[0])[ms]
        s_c, w_c, d_c = O.circle_spectra(k, 1.0, ms)
        errs[N] = [np.abs(np.fft.fft(m[op][0])[ms] / g - ref) / np.abs(ref)
                   for op, ref in (("S", s_c), ("W", w_c), ("D", d_c))]
    for i in range(3):
        ratio = errs[64][i] / errs[128][i]
        assert np.all(ratio > 3.5) and np.all(ratio < 5.0), (i, ratio)
        assert np.all(errs[128][i] < 2e-3)


def test_calderon_identity_circle():
    """S N = I/4 + compact: the continuous product of the circle spectra tends to 1/4,
    and the discrete Z_x = G^-1 S G^-1 N clusters at 1/4 for 1 << |m| << N."""
    k = 1.0
    s_c, w_c, _ = O.circle_spectra(k, 1.0, np.array([20, 40, 80]))
    assert np.all(np.abs(s_c * w_c - 0.25) < np.array([2e-3, 5e-4, 1.5e-4]))
    N = 256
    v = I.regular_polygon(N)
    m = O.assemble(v, k, "SW")
    G = O.gram(v)
    Zx = np.linalg.solve(G, m["S"]) @ np.linalg.solve(G, m["W"])
    z = np.fft.fft(Zx[0])
    assert np.all(np.abs(z[10:30] - 0.25) < 5e-3)
    # away from the cluster: the low-frequency m = 0 mode is not near 1/4
    assert abs(z[0] - 0.25) > 0.1


def test_laplace_limit_constant():
    """As k -> 0, S(k) = S_Laplace + c(k) m m^T + O(k^2) with c(k) = i/4 - (ln(k/2)+gamma)/(2 pi)
    and m_i = int phi_i (DLMF 10.8.2); the difference of two small k isolates c."""
    v, _, _ = I.equal_chord_mesh(I.cos_star(1.0, 0.3, 5), 40)
    mesh = O.Mesh(v)
    k1, k2 = 1e-6, 1e-5
    S1 = O.assemble(v, k1, "S")["S"]
    S2 = O.assemble(v, k2, "S")["S"]
    mvec = 0.5 * (mesh.h + np.roll(mesh.h, 1))
    c = lambda k: 0.25j - (math.log(k / 2) + np.euler_gamma) / (2 * math.pi)
    pred = (c(k1) - c(k2)) * np.outer(mvec, mvec)
    assert np.max(np.abs((S1 - S2) - pred)) <= 1e-8 * np.max(np.abs(pred))


def test_rhs_divergence_theorem():
    """sum_i f_i = -int_Gamma du/dnu = -int_Omega Lap u = k^2 int_Omega u (sum_i phi_i = 1),
    with the area integral over the polygon done by a triangle fan and collapsed Gauss."""
    for verts in (I.regular_polygon(48), I.equal_chord_mesh(I.cos_star(1.0, 0.3, 5), 64)[0]):
        k = 1.7
        ang = np.array([0.0, 0.9, 2.5])
        f = O.rhs_planewave(verts, k, ang)
        xs, ws = O.gauss01(24)
        U, V = np.meshgrid(xs, xs, indexing="ij")
        W2 = np.outer(ws, ws) * U                                # collapsed-square Jacobian
        P1 = np.roll(verts, -1, axis=0)
        area = []
        for phi in ang:
            d = np.array([math.cos(phi), math.sin(phi)])
            tot = 0j
            for a_, b_ in zip(verts, P1):
                # triangle (0, a, b): x = U (a + V (b - a))
                pts = U[..., None] * (a_[None, None, :] + V[..., None] * (b_ - a_)[None, None, :])
                jac = abs(a_[0] * b_[1] - a_[1] * b_[0])
                tot += jac * np.sum(W2 * np.exp(1j * k * (pts @ d)))
            area.append(tot)
        area = np.array(area)
        assert np.allclose(f.sum(axis=0), k * k * area, rtol=1e-13, atol=0)


# ------------------------------------------------------------------ filter, compression, solve


def test_filter_projector_properties(star_case):
    v, _, _ = star_case
    N = v.shape[0]
    n = 21
    P, lam = O.filter_literal(v, n)
    assert np.allclose(P @ P, P, atol=1e-12)
    assert np.allclose(P, P.T, atol=1e-13)
    assert abs(np.trace(P) - n) < 1e-10
    G = O.gram(v)
    Gm = np.linalg.inv(np.linalg.cholesky(G))
    # P commutes with L~; equal chords make P the projector on the Fourier modes |m| <= 10
    Q = O.fourier_basis(N, 10)
    assert np.allclose(P, Q @ Q.T, atol=1e-9)
    Pk, _ = O.filter_literal(v, n, include_kernel=False)
    assert abs(np.trace(Pk) - (n - 1)) < 1e-10
    # the Fourier eigenvalues of the equal-chord Gram matrix
    g = O.gram_eigs(N, float(np.mean(O.Mesh(v).h)), 10)
    assert np.allclose(np.einsum("ij,jk,ki->i", Q.T, G, Q), g, rtol=1e-11)


def test_woodbury_identity():
    rng = np.random.default_rng(5)
    N, r = 50, 7
    U = rng.standard_normal((N, r)) + 1j * rng.standard_normal((N, r))
    Vh = rng.standard_normal((r, N)) + 1j * rng.standard_normal((r, N))
    v = rng.standard_normal((N, 3)) + 1j * rng.standard_normal((N, 3))
    for beta in (0.25, 0.75):
        x = O.woodbury_solve(beta, U * 0.1, Vh * 0.1, v)
        A = beta * np.eye(N) + 0.01 * U @ Vh
        assert np.max(np.abs(A @ x - v)) <= 1e-13 * np.max(np.abs(v))


def test_literal_and_projected_routes_agree(star_case):
    v, k, mats = star_case
    f = O.rhs_planewave(v, k, I.planewave_angles(4))
    lit = O.filtered_solve_literal(mats, v, f, 21, 1e-10)
    pro = O.filtered_solve_projected(mats, v, f, 10, 1e-10)
    assert lit["rank"] == pro["rank"]
    assert np.max(np.abs(lit["x"] - pro["x"])) <= 1e-12 * np.max(np.abs(lit["x"]))
    # rank(P C) <= n
    assert lit["rank"] <= 21
    # the filtered compact part has rank <= n in every representation
    s = np.linalg.svd(lit["PC"], compute_uv=False)
    assert np.all(s[21:] < 1e-13 * s[0])


def test_woodbury_matches_dense_lu(star_case):
    """Uncompressed Woodbury = dense LU of (I/4 + P C2); compressed within tol * kappa."""
    v, k, mats = star_case
    f = O.rhs_planewave(v, k, I.planewave_angles(3))
    lit = O.filtered_solve_literal(mats, v, f, 21, 0.0)
    A = 0.25 * np.eye(v.shape[0]) + lit["PC"]
    kappa = np.linalg.cond(A)
    assert np.max(np.abs(lit["x"] - lit["x_full"])) <= 1e-13 * kappa * np.max(np.abs(lit["x_full"]))
    for tol in (1e-4, 1e-7):
        c = O.filtered_solve_literal(mats, v, f, 21, tol)
        err = np.max(np.abs(c["x"] - c["x_full"])) / np.max(np.abs(c["x_full"]))
        assert err <= 10 * tol * kappa, (tol, err, kappa)
        assert c["rank"] <= lit["rank"]


def test_mie_second_order():
    """The filtered, compressed solution approaches the exact Mie current at O(h^2)."""
    k = 1.0
    errs = []
    for N in (64, 128):
        v = I.regular_polygon(N)
        m = O.assemble(v, k, "SW")
        ang = np.array([0.3, 2.0])
        f = O.rhs_planewave(v, k, ang)
        res = O.filtered_solve_projected(m, v, f, 15, 1e-10)
        G = O.gram(v)
        th = 2 * math.pi * np.arange(N) / N
        e = max(O.g_norm(G, res["x"][:, w] - O.mie_current(k, 1.0, th, ang[w]))[0]
                / O.g_norm(G, O.mie_current(k, 1.0, th, ang[w]))[0] for w in range(2))
        errs.append(e)
    assert errs[1] < 3e-4
    assert 3.5 < errs[0] / errs[1] < 4.6


def test_cfie_filtered_solution_matches_efie():
    """EFIE, MFIE and the Yukawa-Calderon CFIE (Sec. IV-A) describe the same current:
    uncompressed filtered solutions for alpha = 0 and alpha = 1 agree to discretisation
    accuracy, and both approach the Mie current."""
    N, k = 128, 1.0
    v = I.regular_polygon(N)
    m = O.assemble(v, k, "SWD")
    ang = np.array([0.4])
    f = O.rhs_planewave(v, k, ang)
    h2 = O.rhs_planewave_h(v, k, ang)
    e0 = O.filtered_solve_projected(m, v, f, 15, 0.0)
    e1 = O.filtered_solve_projected(m, v, f, 15, 0.0, alpha=1.0, h2=h2)
    th = 2 * math.pi * np.arange(N) / N
    jm = O.mie_current(k, 1.0, th, ang[0])
    G = O.gram(v)
    for res in (e0, e1):
        assert O.g_norm(G, res["x"][:, 0] - jm)[0] / O.g_norm(G, jm)[0] < 1e-3
    assert abs(e1["beta"] - 0.75) < 1e-15


def test_table1_dense_memory_is_complex128():
    """Table I's dense-memory column equals N^2 x 16 bytes: the matrices are complex128,
    the storage the oracle uses."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1.txt")) if l.strip() and not l.startswith("#")]
    for N, _err, dense_mb, _skel in rows:
        N = int(N)
        assert round(N * N * 16 / 1e6) == int(dense_mb) or abs(N * N * 16 / 1e6 - float(dense_mb)) / float(dense_mb) < 0.01
    m = O.assemble(I.regular_polygon(8), 1.0, "S")
    assert m["S"].dtype == np.complex128


# ------------------------------------------------------------------ far field and gradients


def test_farfield_matches_mie_at_second_order():
    """The discrete far field F x of the circle converges to the exact sound-hard far
    field (Mie series) at second order in h: this fixes the constant C0, the sign of the
    Green's representation and the current convention x = -u_tot."""
    k, phi = 1.0, 0.3
    th = np.linspace(0.0, 2 * np.pi, 36, endpoint=False)
    ue = O.mie_farfield(k, 1.0, th, phi)
    errs = []
    for N in (128, 256):
        v = I.regular_polygon(N)
        mats = O.assemble(v, k, "SW")
        x = np.linalg.solve(mats["W"], O.rhs_planewave(v, k, [phi]))
        u = (O.farfield_matrix(v, k, th) @ x)[:, 0]
        errs.append(np.max(np.abs(u - ue)) / np.max(np.abs(ue)))
    assert errs[0] < 5e-4
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_farfield_reciprocity(star_case):
    """u_inf(xhat; d) = u_inf(-d; -xhat): exact for the discrete unfiltered problem, since
    F(xhat) = C0 f(-xhat)^T and N is complex symmetric."""
    v, k, mats = star_case
    angs = np.array([0.2, 1.1, 2.5, 4.0])
    f = O.rhs_planewave(v, k, angs)
    x = np.linalg.solve(mats["W"], f)
    U = O.farfield_matrix(v, k, angs + np.pi) @ x     # U[o, w] = u_inf(-d_o; d_w)
    # u_inf(xhat = d_o + pi; d_w) must equal u_inf(xhat = d_w + pi; d_o)
    assert np.max(np.abs(U - U.T)) <= 1e-11 * np.max(np.abs(U))


def test_misfit_gradients_match_finite_differences(star_case):
    """The adjoint gradients of the far-field misfit against central differences
    (h = 1e-6) of the misfit itself, for the amplitudes (real and imaginary directions)
    and for the preconditioned right-hand side (a random direction)."""
    v, k, mats = star_case
    f = O.rhs_planewave(v, k, np.array([0.0, 2.0, 4.0]))
    route = O.filtered_solve_projected(mats, v, f, 10, 1e-10)
    th = np.linspace(0.0, 2 * np.pi, 24, endpoint=False)
    F = O.farfield_matrix(v, k, th)
    rng = np.random.default_rng(7)
    a = np.array([1.0 + 0.2j, 0.7 - 0.1j, -0.4 + 0.9j])
    target = 0.01 * (rng.standard_normal((len(th), 3)) + 1j * rng.standard_normal((len(th), 3)))
    res = O.misfit_and_gradients(route, F, a, target)
    h = 1e-6
    for w in range(3):
        for unit in (1.0, 1j):
            ap, am = a.copy(), a.copy()
            ap[w] += h * unit
            am[w] -= h * unit
            fd = (O.misfit_and_gradients(route, F, ap, target)["J"] -
                  O.misfit_and_gradients(route, F, am, target)["J"]) / (2 * h)
            g = res["grad_a"][w].real if unit == 1.0 else res["grad_a"][w].imag
            assert abs(fd - g) <= 1e-6 * max(1.0, abs(g)), (w, unit, fd, g)
    # direction dv in the right-hand sides
    dv = rng.standard_normal(route["vx"].shape) + 1j * rng.standard_normal(route["vx"].shape)
    def J_of(vx):
        r2 = dict(route)
        r2["vx"] = vx
        return O.misfit_and_gradients(r2, F, a, target)["J"]
    fd = (J_of(route["vx"] + h * dv) - J_of(route["vx"] - h * dv)) / (2 * h)
    pred = float(np.sum((np.conj(res["grad_v"]) * dv).real))
    assert abs(fd - pred) <= 1e-6 * max(1.0, abs(pred))


# ------------------------------------------------------------------ block route (large meshes)


def test_assemble_entries_matches_assemble(star_case):
    """assemble_entries (the four segment pairs around (i, j), used on the large meshes)
    gives every entry of the dense assembly, for S, N and D."""
    v40, _, _ = I.equal_chord_mesh(I.cos_star(1.0, 0.3, 5), 40)
    k = 1.7
    mats = O.assemble(v40, k, "SWD")
    rows, cols = np.meshgrid(np.arange(40), np.arange(40), indexing="ij")
    ent = O.assemble_entries(v40, k, rows.ravel(), cols.ravel(), "SWD")
    for op in "SWD":
        err = np.max(np.abs(ent[op] - mats[op].ravel())) / np.max(np.abs(mats[op]))
        assert err <= 1e-15, (op, err)


def test_assemble_parallel_blocks_equal_serial():
    v, _, _ = I.equal_chord_mesh(I.cos_star(1.0, 0.3, 5), 37)
    a = O.assemble(v, 1.1, "SWD", block=37)
    b = O.assemble(v, 1.1, "SWD", workers=2, block=5)
    for op in "SWD":
        assert np.max(np.abs(a[op] - b[op])) <= 1e-15 * np.max(np.abs(a[op]))


def test_gram_powers_match_dense():
    """G^-1 and G^-1/2 of the equal-chord Gram matrix by its DFT eigenvalues equal the dense
    solve and the dense symmetric square root of G (Sec. III-A, G^-1/2)."""
    v, _, h = I.equal_chord_mesh(I.random_star(4), 50)
    G = O.gram(v)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((50, 3)) + 1j * rng.standard_normal((50, 3))
    hh = O.chord_length(v)
    assert abs(hh - h) <= 1e-14 * h
    assert np.max(np.abs(O.gram_power_cols(X, hh, -1.0) - np.linalg.solve(G, X))) <= 1e-12 * np.max(np.abs(X)) / hh
    w, V = np.linalg.eigh(G)
    Gm12 = (V * w ** -0.5) @ V.T
    assert np.max(np.abs(O.gram_power_cols(X, hh, -0.5) - Gm12 @ X)) <= 1e-12 * np.max(np.abs(Gm12 @ X))
    assert np.max(np.abs(O.gram_power_rows(X.T, hh, -0.5) - X.T @ Gm12)) <= 1e-12 * np.max(np.abs(Gm12 @ X))
    assert np.allclose(np.sort(O.gram_dft_eigs(50, hh)), w, rtol=1e-13, atol=0)


@pytest.fixture(scope="module")
def star384():
    v, _, _ = I.equal_chord_mesh(I.random_star(2), 384)
    k = 2.0
    return v, k, O.assemble(v, k, "SWD", workers=4)


@pytest.mark.parametrize("alpha,tol", [(0.0, 1e-10), (0.0, 1e-4), (0.5, 1e-10)])
def test_block_route_matches_literal(star384, alpha, tol):
    """The block route (n x N block B, FFT Gram powers, 2n x 2n condition number) reproduces
    the literal route of the paper (dense G^-1/2, eigenvectors of L~, the full N x N Z and
    P C2, Sec. III-A / IV) on a 384-vertex random star, EFIE and CFIE."""
    v, k, mats = star384
    ang = I.planewave_angles(5)
    f = O.rhs_planewave(v, k, ang)
    h2 = O.rhs_planewave_h(v, k, ang) if alpha else None
    M = 20
    lit = O.filtered_solve_literal(mats, v, f, 2 * M + 1, tol, alpha=alpha, h2=h2)
    blk = O.filtered_solve_blocks(mats, v, f, M, tol, alpha=alpha, h2=h2)
    assert blk["rank"] == lit["rank"]
    n = 2 * M + 1
    assert np.max(np.abs(blk["sigma"] - lit["sigma"][:n])) <= 1e-12 * lit["sigma"][0]
    assert np.all(lit["sigma"][n:] <= 1e-13 * lit["sigma"][0])
    for key in ("x", "x_full"):
        err = np.max(np.abs(blk[key] - lit[key])) / np.max(np.abs(lit[key]))
        assert err <= 1e-12, (key, err)
    # x-coordinate right-hand side and the condition number of the filtered operator
    assert np.max(np.abs(blk["vx"] - lit["Gmh"] @ lit["v2"])) <= 1e-12 * np.max(np.abs(blk["vx"]))
    A2 = lit["beta"] * np.eye(v.shape[0]) + lit["PC"]
    kd = np.linalg.cond(A2)
    assert abs(blk["kappa"] - kd) <= 1e-9 * kd, (blk["kappa"], kd)
    # B against the projected route's x-coordinate block (formed there as Q^T G^-1/2 C2 G^1/2
    # from dense square roots, which costs about two more digits of rounding)
    pro = O.filtered_solve_projected(mats, v, f, M, tol, alpha=alpha, h2=h2)
    assert np.max(np.abs(blk["B"] - pro["B"])) <= 1e-11 * np.max(np.abs(pro["B"]))


def test_pointsource_rhs_divergence_theorem():
    """Line source outside the curve: u = g2(|x - r0|) solves the Helmholtz equation inside,
    so sum_i f_i = -int_Gamma du/dnu = k^2 int_Omega u over the polygon (triangle fan,
    collapsed Gauss); and <phi, u> sums to the boundary integral of u."""
    for verts in (I.regular_polygon(48), I.equal_chord_mesh(I.cos_star(1.0, 0.3, 5), 64)[0]):
        k = 1.7
        src = np.array([[3.0, 0.0], [-1.2, 2.5]])
        f = O.rhs_pointsource(verts, k, src)
        xs, ws = O.gauss01(24)
        U, V = np.meshgrid(xs, xs, indexing="ij")
        W2 = np.outer(ws, ws) * U
        P1 = np.roll(verts, -1, axis=0)
        area = []
        for r0 in src:
            tot = 0j
            for a_, b_ in zip(verts, P1):
                pts = U[..., None] * (a_[None, None, :] + V[..., None] * (b_ - a_)[None, None, :])
                jac = abs(a_[0] * b_[1] - a_[1] * b_[0])
                tot += jac * np.sum(W2 * O.green(k, np.linalg.norm(pts - r0, axis=-1)))
            area.append(tot)
        assert np.allclose(f.sum(axis=0), k * k * np.array(area), rtol=1e-12, atol=0)


def test_pointsource_rhs_is_the_planewave_limit():
    """Far away, the line source looks like a plane wave: g2(|x - R d|) ~ C0 e^{ikR}/sqrt(R)
    e^{-ik d.x} (large-argument Hankel form), so the source at R(cos p, sin p) gives the
    plane wave travelling along -(cos p, sin p), times C0 e^{ikR}/sqrt(R), to O(1/R)."""
    verts = I.equal_chord_mesh(I.cos_star(1.0, 0.3, 5), 64)[0]
    k, p = 1.3, 0.7
    errs = []
    for R in (1e3, 1e4):
        src = R * np.array([[math.cos(p), math.sin(p)]])
        fp = O.rhs_pointsource(verts, k, src)[:, 0]
        fw = O.rhs_planewave(verts, k, [p + math.pi])[:, 0]
        scale = O.farfield_constant(k) * np.exp(1j * k * R) / math.sqrt(R)
        errs.append(np.max(np.abs(fp - scale * fw)) / np.max(np.abs(scale * fw)))
    assert errs[1] < 2e-3 and 7 < errs[0] / errs[1] < 13, errs


def test_fig2_spectral_claims_on_the_ellipse():
    """Fig. 2 (Sec. V), ellipse 1.42 x 1.32, k = 0.4, line source at (3, 0), filtering point
    21: projected on the singular vectors q_m of the filter (eigenvectors of L~, smoothest
    first), (a) the compact part C2 grows with the index (the discretisation's spectral
    deviation), (b) the filtered part P C2 has no component beyond the n kept modes, and
    (c) the right-hand side is band-limited with respect to the filter."""
    N, k, n = 128, 0.4, 21
    v, _, _ = I.equal_chord_mesh(I.ellipse(1.42, 1.32), N)
    mats = O.assemble(v, k, "SW")
    f = O.rhs_pointsource(v, k, [[3.0, 0.0]])
    G, L = O.gram(v), O.laplacian(v)
    Z2, v2, Gh, Gmh = O.calderon_system(mats, G, f)
    C2 = Z2 - np.eye(N) / 4.0
    lam, V = np.linalg.eigh(Gmh @ L @ Gmh)
    p = np.linalg.norm(V.T @ C2, axis=1)
    # past the lowest few modes (where the low-frequency part of C2 is O(ka)^2) the projected
    # magnitude grows with the index, by about two orders towards the mesh's Nyquist end
    assert np.mean(p[N // 2:]) > 30.0 * np.mean(p[8:n]), (np.mean(p[N // 2:]), np.mean(p[8:n]))
    assert np.all(np.diff(p[8:N // 2:8]) > 0)
    P, _ = O.filter_literal(v, n)
    pf = np.linalg.norm(V.T @ (P @ C2), axis=1)
    assert np.max(pf[n:]) <= 1e-12 * np.max(pf)
    pv = np.abs(V.T @ v2[:, 0])
    assert np.max(pv[n:]) <= 1e-3 * np.max(pv)
    assert np.max(pv[3 * n:]) <= 1e-11 * np.max(pv)
    assert np.linalg.norm(v2[:, 0] - P @ v2[:, 0]) <= 1e-4 * np.linalg.norm(v2[:, 0])


def test_hypersingular_null_space_at_low_frequency():
    """Maue's form: the derivative term of N has vanishing row sums (sum_b sigma_b = 0), so
    N 1 equals the k^2 term -k^2 sum <phi_i, (nu_x . nu_y) g2 phi_j> exactly.  At k = 1e-3 that
    row sum is O(k^2) of the entries' segment-pair means, so it survives only if the
    derivative term is formed without rounding the means against each other (the exact
    second difference)."""
    N, k = 256, 1e-3
    v, _, _ = I.equal_chord_mesh(I.cos_star(1.0, 0.3, 5), N)
    W = O.assemble(v, k, "W")["W"]
    mesh = O.Mesh(v)
    E, F = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    E, F = E.ravel(), F.ravel()
    Iq, _, _ = O.pair_integrals(mesh, k, E, F, False)
    nud = np.einsum("pc,pc->p", mesh.nu[E], mesh.nu[F])
    K1 = np.zeros(N, dtype=np.complex128)
    for a in range(2):
        np.add.at(K1, (E + a) % N, -(k * k) * nud * Iq[:, a, :].sum(axis=1))
    err = np.max(np.abs(W.sum(axis=1) - K1)) / np.max(np.abs(K1))
    assert err <= 1e-7, err


# ------------------------------------------------------------------ non-equal-chord meshes


def test_general_mesh_gram_and_laplacian_forms():
    """On a graded mesh G and L are the P1 mass and stiffness matrices: G 1 sums to the
    hat integrals (h_{i-1} + h_i)/2, 1^T G 1 is the perimeter, L has the constant kernel,
    and x^T L x of the nodal values of a linear function f(x, y) = c . r equals the
    chord-wise sum of (c . t_e)^2 h_e (the exact energy of the interpolant)."""
    v, _ = I.parameter_mesh(I.perturbed_circle(), 97, grade=0.4)
    h = np.linalg.norm(np.roll(v, -1, 0) - v, axis=1)
    G, L = O.gram(v), O.laplacian(v)
    assert np.allclose(G @ np.ones(97), 0.5 * (h + np.roll(h, 1)), rtol=1e-14)
    assert abs(np.ones(97) @ G @ np.ones(97) - h.sum()) < 1e-13 * h.sum()
    assert np.max(np.abs(L @ np.ones(97))) < 1e-12 * np.max(np.abs(L))
    c = np.array([0.7, -1.3])
    x = v @ c
    t = (np.roll(v, -1, 0) - v) / h[:, None]
    assert abs(x @ L @ x - np.sum((t @ c) ** 2 * h)) < 1e-12 * np.sum((t @ c) ** 2 * h)


def test_general_mesh_filter_is_the_generalized_eigenspace():
    """The literal filter built from L~ = G^-1/2 L G^-1/2 (Sec. III-A) on a graded,
    asymmetric mesh projects onto G^1/2 span(Phi), Phi the n lowest eigenvectors of the
    pencil L phi = lambda G phi from a Cholesky-based generalized solver, with the same
    eigenvalues; the lowest eigenvalues approach those of the curve's Laplace-Beltrami
    operator, (2 pi m / perimeter)^2, at second order in h."""
    sla = pytest.importorskip("scipy.linalg")
    v, _ = I.parameter_mesh(I.perturbed_circle(), 160, grade=0.25, phase=0.7)
    G, L = O.gram(v), O.laplacian(v)
    n = 21
    P, lam = O.filter_literal(v, n)
    w, Phi = sla.eigh(L, G, subset_by_index=[0, n - 1])
    Gh = sla.sqrtm(G).real
    P2 = Gh @ Phi @ Phi.T @ Gh
    assert np.max(np.abs(P - P2)) < 1e-10
    assert np.allclose(lam[:n], w, rtol=1e-10, atol=1e-10)
    errs = []
    for N in (200, 400):
        vv, _ = I.parameter_mesh(I.circle(1.0), N, grade=0.3)
        ww = sla.eigh(O.laplacian(vv), O.gram(vv), eigvals_only=True, subset_by_index=[0, 10])
        m = np.array([0, 1, 1, 2, 2, 3, 3, 4, 4, 5, 5], dtype=float)
        perim = np.linalg.norm(np.roll(vv, -1, 0) - vv, axis=1).sum()
        errs.append(np.max(np.abs(ww - (2 * math.pi * m / perim) ** 2)))
    assert errs[1] < 0.02 and 3.5 < errs[0] / errs[1] < 4.6, errs     # lambda up to 25


def test_general_mesh_mie_second_order():
    """On graded meshes of the unit circle the literal route's filtered, compressed
    solution approaches the exact Mie current at O(h^2), as on equal-chord meshes."""
    k = 1.0
    errs = []
    for N in (64, 128):
        v, th = I.parameter_mesh(I.circle(1.0), N, grade=0.3, phase=0.4)
        m = O.assemble(v, k, "SW")
        ang = np.array([0.3, 2.0])
        f = O.rhs_planewave(v, k, ang)
        res = O.filtered_solve_literal(m, v, f, 15, 1e-10)
        G = O.gram(v)
        e = max(O.g_norm(G, res["x"][:, w] - O.mie_current(k, 1.0, th, ang[w]))[0]
                / O.g_norm(G, O.mie_current(k, 1.0, th, ang[w]))[0] for w in range(2))
        errs.append(e)
    assert errs[1] < 1e-3, errs
    assert 3.3 < errs[0] / errs[1] < 4.8, errs
