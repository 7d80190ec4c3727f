"""CPU FP64 oracle for the filtered Calderon TE-EFIE fast direct solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` do.  It shares no code with the CUDA path.

It is a plain, slow, direct statement of the method of

    Henry, Consoli, Dely, Rahmouni, Merlini, Andriulli,
    "Fast Direct Solvers for Integral Equations at Low-Frequency Based on
    Operator Filtering" (EuCAP 2023, arXiv 2210.08580),

in numpy/scipy double precision, following the paper's order:

  Sec. II   g2 = (i/4) H0^(1)(k r); the operators S, N (hypersingular) and D;
            P1 hats phi_i, Galerkin matrices [X]_ij = <phi_i, X phi_j>, Gram G,
            the normalised Calderon TE-EFIE  Z2 j2 = v_e2 (with the reading that
            the preconditioner carries the factor i k, see ``calderon_system``),
            C2 = Z2 - I/4.
  Sec. III  Laplacian L, L~ = G^-1/2 L G^-1/2, the filter P^L_n from the n
            smoothest eigenvectors of L~ (eq. LapFilter).  The literal route
            (``filter_literal``, ``filtered_solve_literal``) takes any mesh, including
            the non-equal-chord ones for which the paper prescribes L~; the block route
            is for equal-chord meshes, where G and L are circulant.
  Sec. IV   filtered equation (I/4 + P C2) j2 = v_e2, its CFIE generalisation,
            low-rank C = U V^H and the Woodbury inverse.

Readings of points the paper leaves open (each is listed with its reason in the
project's design notes):
  * the hypersingular Galerkin matrix uses Maue's integration by parts,
        <phi_i, N phi_j> = int int g [phi_i'(x) phi_j'(y) - k^2 (nu_x.nu_y) phi_i(x) phi_j(y)];
  * the incident field is u_inc = H_z^inc = exp(i k d.x) and the EFIE right-hand side
    is f_i = -<phi_i, d u_inc/d nu>, so that N x = f (Sec. II, eq. TE-EFIE times i k);
  * the filter keeps the n = 2M+1 smoothest modes *including* the constant (kernel)
    mode by default; ``include_kernel=False`` gives the literal L_n^+ L_n;
  * the compression tolerance is relative to the largest singular value of the
    filtered compact part in the orthonormal (G^1/2-weighted) basis.

Quadrature (the paper does not specify one) is the oracle's own and is deliberately
different from the CUDA path's: converged high-order tensor Gauss-Legendre on
separated segment pairs, a difference-variable substitution with geometrically
graded Gauss on self pairs, and a Duffy split with graded Gauss on adjacent pairs.
Bessel functions come from scipy.special (Cephes j0/y0/j1/y1).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

__all__ = [
    "Mesh", "green", "green_dnu_factor", "gauss01", "graded_gauss01",
    "pair_integrals", "assemble", "assemble_entries", "gram", "laplacian",
    "rhs_planewave", "rhs_planewave_h", "rhs_pointsource", "rhs_pointsource_h", "fourier_basis", "gram_eigs", "filter_literal",
    "calderon_system", "filtered_solve_literal", "filtered_solve_projected",
    "woodbury_solve", "mie_current", "circle_spectra", "g_norm",
    "farfield_constant", "farfield_matrix", "mie_farfield", "misfit_and_gradients",
    "chord_length", "gram_dft_eigs", "gram_power_rows", "gram_power_cols", "filtered_block",
    "compress_block", "filtered_condition", "filtered_solve_blocks", "assembled_column_blocks",
    "segment_pair_means", "maue_second_difference", "misfit_blocks",
]

# --------------------------------------------------------------------------------------
# Green's function and its normal derivative (Sec. II)
# --------------------------------------------------------------------------------------


def green(k: float, r):
    """g2(r) = (i/4) H0^(1)(k r) = (i/4)(J0 + i Y0)."""
    z = k * np.asarray(r, dtype=np.float64)
    return 0.25j * special.j0(z) - 0.25 * special.y0(z)


def green_dnu_factor(k: float, r):
    """-(i k/4) H1^(1)(k r) / r, so that d g2(x,y)/d nu_y = factor * ((y - x).nu_y)."""
    r = np.asarray(r, dtype=np.float64)
    z = k * r
    return (-0.25j * k) * (special.j1(z) + 1j * special.y1(z)) / r


# --------------------------------------------------------------------------------------
# Mesh
# --------------------------------------------------------------------------------------


class Mesh:
    """N vertices (counter-clockwise), N segments e = [r_e, r_{e+1 mod N}].

    h_e segment length, t_e unit tangent, nu_e = (t_y, -t_x) outward unit normal.
    P1 hat phi_i is 1 at vertex i: on segment e its local shape functions are
    lambda_0(s) = 1 - s/h_e (vertex e) and lambda_1(s) = s/h_e (vertex e+1).
    """

    def __init__(self, verts):
        v = np.ascontiguousarray(np.asarray(verts, dtype=np.float64))
        assert v.ndim == 2 and v.shape[1] == 2 and v.shape[0] >= 3
        self.verts = v
        self.N = v.shape[0]
        self.P0 = v
        self.P1 = np.roll(v, -1, axis=0)
        d = self.P1 - self.P0
        self.h = np.linalg.norm(d, axis=1)
        self.t = d / self.h[:, None]
        self.nu = np.stack([self.t[:, 1], -self.t[:, 0]], axis=1)


# --------------------------------------------------------------------------------------
# Quadrature rules
# --------------------------------------------------------------------------------------


def gauss01(q: int):
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def graded_gauss01(ratio: float = 0.3, q: int = 16, levels: int = 34):
    """Composite Gauss-Legendre on [0,1] with intervals [ratio^{j+1}, ratio^j],
    j = 0..levels-1, plus [0, ratio^levels]: resolves integrable endpoint
    singularities (log, x log x) at 0."""
    xs, ws = gauss01(q)
    nodes, weights = [], []
    hi = 1.0
    for _ in range(levels):
        lo = hi * ratio
        nodes.append(lo + (hi - lo) * xs)
        weights.append((hi - lo) * ws)
        hi = lo
    nodes.append(hi * xs)
    weights.append(hi * ws)
    return np.concatenate(nodes), np.concatenate(weights)


def _q_for_gap(gap_over_h, k_gap):
    """Gauss order from the Bernstein-ellipse bound rho^{-2q} exp(k Im r) <= 1e-20 for the
    kernel on a segment pair: rho for a singularity at distance ``gap`` beyond the end of a
    unit-normalised segment, and the Hankel kernel grows like exp(k Im r) off the real
    axis, where Im r reaches about the gap (``k_gap`` = k (gap + h)); one point of margin."""
    a = 1.0 + 2.0 * np.maximum(gap_over_h, 1e-3)
    rho = a + np.sqrt(a * a - 1.0)
    q = np.ceil((20.0 * math.log(10.0) + k_gap) / (2.0 * np.log(rho))) + 1
    return np.clip(q, 4, 60).astype(int)


def _seg_seg_gap(mesh: Mesh, e, f):
    """Minimum distance between segments e and f (non-intersecting), vectorised."""
    def pt_seg(p, a, b):
        ab = b - a
        tt = np.clip(np.einsum("ij,ij->i", p - a, ab) / np.einsum("ij,ij->i", ab, ab), 0.0, 1.0)
        return np.linalg.norm(p - (a + tt[:, None] * ab), axis=1)
    A0, A1, B0, B1 = mesh.P0[e], mesh.P1[e], mesh.P0[f], mesh.P1[f]
    return np.minimum.reduce([pt_seg(A0, B0, B1), pt_seg(A1, B0, B1),
                              pt_seg(B0, A0, A1), pt_seg(B1, A0, A1)])


# --------------------------------------------------------------------------------------
# Local integrals of one segment pair
#   I[a,b]  = int_e int_f lambda_a(s) g2(|x-y|) lambda_b(t) dt ds
#   J[a,b]  = same with d g2/d nu_y  (normal on f; D's kernel, Sec. II)
#   Jt[a,b] = same with d g2(y,x)/d nu_x  (normal on e; used for D's transpose)
# --------------------------------------------------------------------------------------


def _moments(k, x, y, wx, wy, lam_x, lam_y, nu_e, nu_f, scale, need_d):
    """Tensor quadrature moments over points x (P,qx,2), y (P,qy,2)."""
    diff = y[:, None, :, :] - x[:, :, None, :]                 # (P,qx,qy,2)  y - x
    r = np.linalg.norm(diff, axis=-1)
    w = wx[:, :, None] * wy[:, None, :] * scale[:, None, None]
    g = green(k, r) * w
    I = np.einsum("pst,pas,pbt->pab", g, lam_x, lam_y)
    if not need_d:
        return I, None, None
    fac = green_dnu_factor(k, r) * w
    dn_f = np.einsum("pstc,pc->pst", diff, nu_f)               # (y - x).nu_f
    dn_e = -np.einsum("pstc,pc->pst", diff, nu_e)              # (x - y).nu_e
    J = np.einsum("pst,pas,pbt->pab", fac * dn_f, lam_x, lam_y)
    Jt = np.einsum("pst,pas,pbt->pab", fac * dn_e, lam_x, lam_y)
    return I, J, Jt


def _pairs_far(mesh: Mesh, k, e, f, q, need_d):
    s, ws = gauss01(q)
    P = len(e)
    x = mesh.P0[e][:, None, :] + (mesh.h[e][:, None] * s[None, :])[..., None] * mesh.t[e][:, None, :]
    y = mesh.P0[f][:, None, :] + (mesh.h[f][:, None] * s[None, :])[..., None] * mesh.t[f][:, None, :]
    lam = np.stack([1.0 - s, s])                               # (2,q)
    lam = np.broadcast_to(lam, (P, 2, q))
    wq = np.broadcast_to(ws, (P, q))
    return _moments(k, x, y, wq, wq, lam, lam, mesh.nu[e], mesh.nu[f],
                    mesh.h[e] * mesh.h[f], need_d)


def _pairs_self(mesh: Mesh, k, e, need_d):
    """Self pair: with u = |s - t| the double integral becomes
    int_0^h g2(u) w_ab(u) du, w_ab(u) = int_0^{h-u} [l_a(t+u) l_b(t) + l_a(t) l_b(t+u)] dt,
    the inner integral exact by 3-point Gauss (quadratic in t); the outer is log-singular
    at u = 0 and is integrated on a geometrically graded mesh.  D's kernel vanishes on a
    flat segment ((y - x).nu = 0)."""
    e = np.asarray(e)
    P = len(e)
    h = mesh.h[e]
    uu, wu = graded_gauss01()
    t3, w3 = gauss01(3)
    I = np.zeros((P, 2, 2), dtype=np.complex128)
    for p in range(P):
        hp = h[p]
        u = hp * uu
        L = hp - u                                             # length of the t range
        t = L[:, None] * t3[None, :]                           # (nu, 3)
        wt = L[:, None] * w3[None, :]
        lam = lambda a, s: (1.0 - s / hp) if a == 0 else (s / hp)
        g = green(k, u) * (hp * wu)
        for a in range(2):
            for b in range(2):
                wab = np.sum(wt * (lam(a, t + u[:, None]) * lam(b, t) + lam(a, t) * lam(b, t + u[:, None])), axis=1)
                I[p, a, b] = np.sum(g * wab)
    Z = np.zeros_like(I) if need_d else None
    return I, Z, (np.zeros_like(I) if need_d else None)


def _pairs_adjacent_fwd(mesh: Mesh, k, e, f, need_d):
    """f follows e (shared vertex P = end of e = start of f).  With u = sigma/h_e
    (x = P - sigma t_e) and v = tau/h_f (y = P + tau t_f) the square [0,1]^2 is split
    along u = v and each triangle is mapped by Duffy coordinates (rho, w) with
    Jacobian rho; the log singularity at rho = 0 is integrated with graded Gauss in
    rho and plain Gauss in w."""
    e = np.asarray(e); f = np.asarray(f)
    P = len(e)
    rr, wr = graded_gauss01()
    ww, wwq = gauss01(24)
    RHO, WW = np.meshgrid(rr, ww, indexing="ij")
    WR = wr[:, None] * wwq[None, :] * RHO                      # includes Jacobian rho
    pts = []
    for tri in range(2):
        if tri == 0:
            U, V = RHO, RHO * WW                                # v <= u
        else:
            U, V = RHO * WW, RHO                                # u <  v
        pts.append((U.ravel(), V.ravel(), WR.ravel()))
    U = np.concatenate([p[0] for p in pts]); V = np.concatenate([p[1] for p in pts])
    Wt = np.concatenate([p[2] for p in pts])
    # y - x = sigma t_e + tau t_f, formed directly (no cancellation near the vertex)
    diff = ((mesh.h[e][:, None] * U[None, :])[..., None] * mesh.t[e][:, None, :]
            + (mesh.h[f][:, None] * V[None, :])[..., None] * mesh.t[f][:, None, :])
    r = np.linalg.norm(diff, axis=-1)
    w = Wt[None, :] * (mesh.h[e] * mesh.h[f])[:, None]
    # local shape functions: on e, s = h_e - sigma, so lambda_0 = u, lambda_1 = 1 - u
    lx = np.stack([U, 1.0 - U])                                # (2, npts)
    ly = np.stack([1.0 - V, V])
    g = green(k, r) * w
    I = np.einsum("pn,an,bn->pab", g, lx, ly)
    if not need_d:
        return I, None, None
    fac = green_dnu_factor(k, r) * w
    J = np.einsum("pn,an,bn->pab", fac * np.einsum("pnc,pc->pn", diff, mesh.nu[f]), lx, ly)
    Jt = np.einsum("pn,an,bn->pab", fac * np.einsum("pnc,pc->pn", -diff, mesh.nu[e]), lx, ly)
    return I, J, Jt


def pair_integrals(mesh: Mesh, k: float, e, f, need_d: bool = True):
    """Local 2x2 integrals (I, J, Jt) for arrays of ordered segment pairs (e, f)."""
    e = np.atleast_1d(np.asarray(e, dtype=np.int64)) % mesh.N
    f = np.atleast_1d(np.asarray(f, dtype=np.int64)) % mesh.N
    P = len(e)
    N = mesh.N
    I = np.zeros((P, 2, 2), dtype=np.complex128)
    J = np.zeros((P, 2, 2), dtype=np.complex128) if need_d else None
    Jt = np.zeros((P, 2, 2), dtype=np.complex128) if need_d else None
    same = e == f
    fwd = (f == (e + 1) % N) & ~same
    bwd = (e == (f + 1) % N) & ~same & ~fwd
    far = ~(same | fwd | bwd)
    if same.any():
        i_, j_, jt_ = _pairs_self(mesh, k, e[same], need_d)
        I[same] = i_
    if fwd.any():
        i_, j_, jt_ = _pairs_adjacent_fwd(mesh, k, e[fwd], f[fwd], need_d)
        I[fwd] = i_
        if need_d:
            J[fwd] = j_; Jt[fwd] = jt_
    if bwd.any():
        # (e, f) with e following f: evaluate (f, e) and swap the roles of the segments
        i_, j_, jt_ = _pairs_adjacent_fwd(mesh, k, f[bwd], e[bwd], need_d)
        I[bwd] = np.swapaxes(i_, 1, 2)
        if need_d:
            J[bwd] = np.swapaxes(jt_, 1, 2)
            Jt[bwd] = np.swapaxes(j_, 1, 2)
    if far.any():
        idx = np.nonzero(far)[0]
        hmx = np.maximum(mesh.h[e[idx]], mesh.h[f[idx]])
        gap = _seg_seg_gap(mesh, e[idx], f[idx])
        qs = _q_for_gap(gap / hmx, k * (gap + hmx))
        for q in np.unique(qs):
            sel = idx[qs == q]
            for c0 in range(0, len(sel), 20000):
                cs = sel[c0:c0 + 20000]
                i_, j_, jt_ = _pairs_far(mesh, k, e[cs], f[cs], int(q), need_d)
                I[cs] = i_
                if need_d:
                    J[cs] = j_; Jt[cs] = jt_
    return I, J, Jt


# --------------------------------------------------------------------------------------
# Galerkin matrices (Sec. II):  S, N (= W here, Maue form) and D
# --------------------------------------------------------------------------------------



def _scatter(mesh, k, e, f, I, J, ops):
    """Vertex-matrix contributions of segment pairs (e, f): i = e + a, j = f + b.  For N
    (Maue's form) only the k^2 term -k^2 (nu_e . nu_f) I_ab is scattered here ('K'); its
    derivative term is kept per segment pair (segment_pair_means) and applied as an exact
    second difference (maue_second_difference)."""
    N = mesh.N
    out = {}
    nudot = np.einsum("pc,pc->p", mesh.nu[e], mesh.nu[f])
    for a in range(2):
        for b in range(2):
            ii = (e + a) % N
            jj = (f + b) % N
            if "S" in ops:
                out.setdefault("S", []).append((ii, jj, I[:, a, b]))
            if "W" in ops:
                out.setdefault("K", []).append((ii, jj, -(k * k) * nudot * I[:, a, b]))
            if "D" in ops:
                out.setdefault("D", []).append((ii, jj, J[:, a, b]))
    return out


def segment_pair_means(mesh, e, f, I):
    """M0(e, f) = int_e int_f g2 / (h_e h_f) = sum_ab I_ab / (h_e h_f): with phi_i' = sigma / h
    on the segments around vertex i, the derivative term of Maue's form for the pair is
    sigma_a sigma_b M0(e, f)."""
    return I.sum(axis=(1, 2)) / (mesh.h[e] * mesh.h[f])


def maue_second_difference(Mg):
    """Derivative term of Maue's form, sum_{a,b} sigma_a sigma_b Mg[i - a, j - b] with
    sigma_0 = -1, sigma_1 = +1 (phi_i' = -1/h on segment i, +1/h on segment i - 1), for the
    N x N matrix of segment-pair means Mg[e, f] = M0(e, f), evaluated as
        (Mg[i-1, j-1] - Mg[i-1, j]) - (Mg[i, j-1] - Mg[i, j]).
    Away from the diagonal the four means agree to many digits, and the difference of two
    close doubles is exact (Sterbenz), so the term's rounding is that of the small
    differences rather than of the means: its row sums, which vanish identically
    (sum_b sigma_b = 0), stay at that level.  At low k the row sums of N are O(k^2) of the
    means and carry the Calderon product's smallest eigenvalue."""
    R = np.roll(Mg, 1, axis=1) - Mg                                # R[e, j] = Mg[e, j-1] - Mg[e, j]
    return np.roll(R, 1, axis=0) - R                               # R[i-1, j] - R[i, j]


def _assemble_columns(verts, k, f0, f1, ops):
    """Contributions of the segment pairs (e, f), every e and f0 <= f < f1, to the vertex
    columns j = f + b, i.e. columns f0 .. f1 (mod N): a dict of N x (f1 - f0 + 1) blocks
    ('S', 'D', and 'K' the k^2 term of N), plus 'Mg' (N x (f1 - f0)), the segment-pair means
    of the segment columns f0 .. f1 - 1."""
    mesh = Mesh(verts)
    N = mesh.N
    nb = f1 - f0 + 1
    keys = [op for op in ops if op != "W"] + (["K"] if "W" in ops else [])
    out = {op: np.zeros((N, nb), dtype=np.complex128) for op in keys}
    if "W" in ops:
        out["Mg"] = np.zeros((N, f1 - f0), dtype=np.complex128)
    e = np.tile(np.arange(N), f1 - f0)
    f = np.repeat(np.arange(f0, f1), N)
    for c0 in range(0, len(e), 200000):
        ec = e[c0:c0 + 200000]; fc = f[c0:c0 + 200000]
        I, J, _ = pair_integrals(mesh, k, ec, fc, "D" in ops)
        for op, lst in _scatter(mesh, k, ec, fc, I, J, ops).items():
            for ii, jj, val in lst:
                # column jj = f + b (mod N) sits at block column f - f0 + b
                np.add.at(out[op], (ii, (jj - f0) % N), val)
        if "W" in ops:
            out["Mg"][ec, fc - f0] = segment_pair_means(mesh, ec, fc, I)
    return out


def assembled_column_blocks(verts, k: float, starts, block: int = 32, ops: str = "SW", workers: int = 1,
                            pool=None):
    """Yields (f0, blocks) for the segment columns f0 .. f0 + block - 1 of each f0 in
    ``starts`` (see _assemble_columns), in order; ``pool`` (a multiprocessing pool) or
    ``workers`` > 1 (a pool started with ``spawn``) spreads the blocks over processes."""
    verts = np.ascontiguousarray(np.asarray(verts, dtype=np.float64))
    N = verts.shape[0]
    jobs = [(verts, k, f0, min(f0 + block, N), ops) for f0 in starts]
    if pool is not None:
        for j, blk in zip(jobs, pool.imap(_assemble_star, jobs)):
            yield j[2], blk
    elif workers <= 1:
        for j in jobs:
            yield j[2], _assemble_columns(*j)
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as p:
            for j, blk in zip(jobs, p.imap(_assemble_star, jobs)):
                yield j[2], blk


def assemble(verts, k: float, ops: str = "SWD", workers: int = 1, block: int = 32, pool=None):
    """Dense Galerkin matrices {'S','W','D'} (complex128, N x N), by looping over all
    ordered segment pairs, in blocks of ``block`` segment columns.  W is the hypersingular
    operator N of the paper.  ``workers`` > 1 (or a ``pool``) spreads the blocks over
    processes; the sum over pairs is the same."""
    verts = np.ascontiguousarray(np.asarray(verts, dtype=np.float64))
    N = verts.shape[0]
    mats = {op: np.zeros((N, N), dtype=np.complex128) for op in ops}
    Mg = np.zeros((N, N), dtype=np.complex128) if "W" in ops else None
    for f0, blk in assembled_column_blocks(verts, k, range(0, N, block), block, ops, workers, pool):
        for op in ops:
            src = blk["K"] if op == "W" else blk[op]                # N: its k^2 term first
            for c in range(src.shape[1]):
                mats[op][:, (f0 + c) % N] += src[:, c]
        if Mg is not None:
            Mg[:, f0:f0 + blk["Mg"].shape[1]] = blk["Mg"]
    if Mg is not None:
        # Maue's form: N = (second difference of the segment-pair means) + k^2 term
        mats["W"] = maue_second_difference(Mg) + mats["W"]
    return mats


def _assemble_star(args):
    return _assemble_columns(*args)


def assemble_entries(verts, k: float, rows, cols, ops: str = "SWD"):
    """Selected entries (i, j) of S, W, D, each from the four segment pairs that
    touch vertices i and j (used to check large matrices entry by entry)."""
    mesh = Mesh(verts)
    N = mesh.N
    rows = np.asarray(rows, dtype=np.int64); cols = np.asarray(cols, dtype=np.int64)
    out = {op: np.zeros(len(rows), dtype=np.complex128) for op in ops}
    need_d = "D" in ops
    M = {}
    for a in range(2):
        for b in range(2):
            e = (rows - a) % N
            f = (cols - b) % N
            I, J, _ = pair_integrals(mesh, k, e, f, need_d)
            nudot = np.einsum("pc,pc->p", mesh.nu[e], mesh.nu[f])
            M[a, b] = segment_pair_means(mesh, e, f, I)               # Mg[i - a, j - b]
            if "S" in ops:
                out["S"] += I[:, a, b]
            if "W" in ops:
                out["W"] += -(k * k) * nudot * I[:, a, b]
            if "D" in ops:
                out["D"] += J[:, a, b]
    if "W" in ops:
        # the derivative term in the order of maue_second_difference
        out["W"] = ((M[1, 1] - M[1, 0]) - (M[0, 1] - M[0, 0])) + out["W"]
    return out


def gram(verts):
    """[G]_ij = <phi_i, phi_j> for P1 hats (cyclic tridiagonal)."""
    mesh = Mesh(verts)
    N = mesh.N
    G = np.zeros((N, N))
    for e in range(N):
        i, j = e, (e + 1) % N
        h = mesh.h[e]
        G[i, i] += h / 3.0; G[j, j] += h / 3.0
        G[i, j] += h / 6.0; G[j, i] += h / 6.0
    return G


def laplacian(verts):
    """[L]_ij = <grad phi_i, grad phi_j> (Sec. III-A), cyclic tridiagonal."""
    mesh = Mesh(verts)
    N = mesh.N
    L = np.zeros((N, N))
    for e in range(N):
        i, j = e, (e + 1) % N
        c = 1.0 / mesh.h[e]
        L[i, i] += c; L[j, j] += c
        L[i, j] -= c; L[j, i] -= c
    return L


def _segment_gauss(mesh, q=16):
    s, ws = gauss01(q)
    x = mesh.P0[:, None, :] + (mesh.h[:, None] * s[None, :])[..., None] * mesh.t[:, None, :]
    return s, ws, x


def rhs_planewave(verts, k: float, angles):
    """f_i = -<phi_i, d u_inc / d nu>, u_inc = exp(i k d.x), d = (cos phi, sin phi).

    Returns f (N, nrhs) complex.  Gauss-Legendre (16 points) per segment; the
    integrand is entire."""
    mesh = Mesh(verts)
    N = mesh.N
    ang = np.asarray(angles, dtype=np.float64)
    d = np.stack([np.cos(ang), np.sin(ang)], axis=1)             # (nrhs, 2)
    s, ws, x = _segment_gauss(mesh)
    phase = np.einsum("eqc,wc->eqw", x, d)                       # (N, q, nrhs)
    dnu = np.einsum("ec,wc->ew", mesh.nu, d)                     # (N, nrhs)
    val = (1j * k) * dnu[:, None, :] * np.exp(1j * k * phase)     # d u_inc / d nu
    wgt = (mesh.h[:, None] * ws[None, :])                        # (N, q)
    f = np.zeros((N, len(ang)), dtype=np.complex128)
    for a, lam in enumerate((1.0 - s, s)):
        contrib = -np.einsum("eq,eqw->ew", wgt * lam[None, :], val)
        f += np.roll(contrib, a, axis=0)                          # vertex e + a
    return f


def rhs_planewave_h(verts, k: float, angles):
    """[h2]_i = <phi_i, h_z^inc> with h_z^inc = u_inc = exp(i k d.x) (TE-MFIE, Sec. II)."""
    mesh = Mesh(verts)
    N = mesh.N
    ang = np.asarray(angles, dtype=np.float64)
    d = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    s, ws, x = _segment_gauss(mesh)
    val = np.exp(1j * k * np.einsum("eqc,wc->eqw", x, d))
    wgt = (mesh.h[:, None] * ws[None, :])
    out = np.zeros((N, len(ang)), dtype=np.complex128)
    for a, lam in enumerate((1.0 - s, s)):
        out += np.roll(np.einsum("eq,eqw->ew", wgt * lam[None, :], val), a, axis=0)
    return out


def rhs_pointsource(verts, k: float, sources):
    """f_i = -<phi_i, d u_inc / d nu> for the line source u_inc(x) = g2(|x - r0|) (the paper's
    2D "dipole" source of Sec. V read as a z-directed line source): d u_inc / d nu =
    green_dnu_factor(k, rho) ((x - r0).nu) with rho = |x - r0|.  Returns (N, nsrc); 16-point
    Gauss-Legendre per segment (the source lies off the curve)."""
    mesh = Mesh(verts)
    N = mesh.N
    src = np.asarray(sources, dtype=np.float64).reshape(-1, 2)
    s, ws, x = _segment_gauss(mesh)
    diff = x[:, :, None, :] - src[None, None, :, :]                  # x - r0, (N, q, nsrc, 2)
    rho = np.linalg.norm(diff, axis=-1)
    val = green_dnu_factor(k, rho) * np.einsum("eqwc,ec->eqw", diff, mesh.nu)
    wgt = (mesh.h[:, None] * ws[None, :])
    f = np.zeros((N, src.shape[0]), dtype=np.complex128)
    for a, lam in enumerate((1.0 - s, s)):
        f += np.roll(-np.einsum("eq,eqw->ew", wgt * lam[None, :], val), a, axis=0)
    return f


def rhs_pointsource_h(verts, k: float, sources):
    """[h2]_i = <phi_i, u_inc> for the line source u_inc = g2(|x - r0|)."""
    mesh = Mesh(verts)
    N = mesh.N
    src = np.asarray(sources, dtype=np.float64).reshape(-1, 2)
    s, ws, x = _segment_gauss(mesh)
    rho = np.linalg.norm(src[None, None, :, :] - x[:, :, None, :], axis=-1)
    val = green(k, rho)
    wgt = (mesh.h[:, None] * ws[None, :])
    out = np.zeros((N, src.shape[0]), dtype=np.complex128)
    for a, lam in enumerate((1.0 - s, s)):
        out += np.roll(np.einsum("eq,eqw->ew", wgt * lam[None, :], val), a, axis=0)
    return out


# --------------------------------------------------------------------------------------
# Laplacian filter (Sec. III-A)
# --------------------------------------------------------------------------------------


def fourier_basis(N: int, M: int, include_kernel: bool = True):
    """Orthonormal real Fourier modes |m| <= M on the vertex index: columns
    [1/sqrt N, sqrt(2/N) cos(2 pi m i/N), sqrt(2/N) sin(2 pi m i/N)] for m = 1..M
    (cos and sin of each m adjacent).  Eigenvectors of every symmetric circulant."""
    i = np.arange(N)
    cols = []
    if include_kernel:
        cols.append(np.full(N, 1.0 / math.sqrt(N)))
    for m in range(1, M + 1):
        cols.append(math.sqrt(2.0 / N) * np.cos(2.0 * math.pi * m * i / N))
        cols.append(math.sqrt(2.0 / N) * np.sin(2.0 * math.pi * m * i / N))
    return np.stack(cols, axis=1)


def gram_eigs(N: int, h: float, M: int, include_kernel: bool = True):
    """Eigenvalues of the equal-chord Gram matrix on the columns of fourier_basis:
    g_m = h (2 + cos(2 pi m / N)) / 3."""
    ms = ([0] if include_kernel else []) + [m for m in range(1, M + 1) for _ in (0, 1)]
    ms = np.array(ms, dtype=np.float64)
    return h * (2.0 + np.cos(2.0 * math.pi * ms / N)) / 3.0


def _sym_pow(A, p):
    w, V = np.linalg.eigh(A)
    return (V * w ** p) @ V.T


def filter_literal(verts, n: int, include_kernel: bool = True):
    """P^L_n from the eigendecomposition of L~ = G^-1/2 L G^-1/2 (eq. LapFilter).

    The n smallest eigenvalues of L~ (the smoothest modes) are kept.  With
    ``include_kernel=False`` the literal L_n^+ L_n drops the zero (constant) mode."""
    G = gram(verts)
    L = laplacian(verts)
    Gm12 = _sym_pow(G, -0.5)
    Lt = Gm12 @ L @ Gm12
    lam, V = np.linalg.eigh(Lt)
    keep = V[:, :n]
    if not include_kernel:
        keep = keep[:, 1:]
    return keep @ keep.T, lam


# --------------------------------------------------------------------------------------
# Calderon system (Sec. II) and the filtered fast direct solver (Sec. IV)
# --------------------------------------------------------------------------------------


def calderon_system(mats, G, f):
    """Normalised Calderon TE-EFIE, Z2 = G^-1/2 S G^-1 N G^-1/2, v2 = G^-1/2 S G^-1 f.

    Reading: the paper's Z2 carries (i k)^-1 and v_e2 does not; the factor is moved to
    the right-hand side (f = -<phi, du_inc/dnu> = i k (-eta^-1 e2)), which makes
    Z2 -> I/4 + compact, as the Calderon identity S N = I/4 + C2 requires."""
    S, W = mats["S"], mats["W"]
    Gh = _sym_pow(G, 0.5)
    Gmh = _sym_pow(G, -0.5)
    Z2 = Gmh @ S @ np.linalg.solve(G, W) @ Gmh
    v2 = Gmh @ S @ np.linalg.solve(G, f)
    return Z2, v2, Gh, Gmh


def woodbury_solve(beta, U, Vh, v):
    """(beta I + U V^H)^-1 v = v/beta - beta^-2 U (I_r + beta^-1 V^H U)^-1 V^H v (Sec. IV-C)."""
    r = U.shape[1]
    K = np.eye(r, dtype=np.complex128) + (Vh @ U) / beta
    return v / beta - (U @ np.linalg.solve(K, Vh @ v)) / (beta * beta)


def _truncate(T, tol):
    Uu, s, Vh = np.linalg.svd(T, full_matrices=False)
    if tol <= 0:
        r = int(np.sum(s > 0))
    else:
        r = int(np.sum(s >= tol * s[0]))
    return Uu[:, :r] * s[:r], Vh[:r, :], s, r


def _compact_parts(mats, G, f, alpha, h2):
    Z2, v2, Gh, Gmh = calderon_system(mats, G, f)
    N = Z2.shape[0]
    C2 = Z2 - np.eye(N) / 4.0
    if alpha != 0.0:
        # normalised TE-MFIE: (I/2 - G^-1/2 D G^-1/2) j2 = v_h2 = -G^-1/2 h2; its compact
        # part relative to I/2 is -G^-1/2 D G^-1/2 (Sec. IV-A, combined as the CFIE).
        Dn = Gmh @ mats["D"] @ Gmh
        C2 = C2 - alpha * Dn
        v2 = v2 + alpha * (-(Gmh @ h2))
    beta = (1.0 + 2.0 * alpha) / 4.0
    return C2, v2, beta, Gh, Gmh


def filtered_solve_literal(mats, verts, f, n, tol, alpha=0.0, h2=None, include_kernel=True):
    """Literal route: dense P^L_n from eig(L~), SVD of P C2, Woodbury (Sec. IV).
    Returns dict with x (nodal coefficients, N x nrhs), j2, rank, sigma, and the
    uncompressed filtered solution x_full (dense LU of beta I + P C2)."""
    G = gram(verts)
    C2, v2, beta, Gh, Gmh = _compact_parts(mats, G, f, alpha, h2)
    P, _ = filter_literal(verts, n, include_kernel)
    PC = P @ C2
    U, Vh, s, r = _truncate(PC, tol)
    j2 = woodbury_solve(beta, U, Vh, v2)
    N = PC.shape[0]
    j2_full = np.linalg.solve(beta * np.eye(N) + PC, v2)
    return dict(x=Gmh @ j2, j2=j2, rank=r, sigma=s, x_full=Gmh @ j2_full, beta=beta,
                PC=PC, C2=C2, v2=v2, U=U, Vh=Vh, Gh=Gh, Gmh=Gmh)


def filtered_solve_projected(mats, verts, f, M, tol, alpha=0.0, h2=None, include_kernel=True):
    """Projected route: P^L_n = Q Q^T with the Fourier basis Q (N x n), which is exact for
    an equal-chord mesh (G and L circulant).  The filtered compact part Q (Q^T C2) is
    compressed through the SVD of the n x N block B^ = Q^T C2.  Also returns
    B = Q^T C_x, C_x = G^-1/2 C2 G^1/2 (the x-coordinate block)."""
    verts = np.asarray(verts)
    N = verts.shape[0]
    G = gram(verts)
    C2, v2, beta, Gh, Gmh = _compact_parts(mats, G, f, alpha, h2)
    Q = fourier_basis(N, M, include_kernel)
    Bhat = Q.T @ C2
    Eu, s, Fh = np.linalg.svd(Bhat, full_matrices=False)
    r = int(np.sum(s >= tol * s[0])) if tol > 0 else int(np.sum(s > 0))
    U2 = Q @ (Eu[:, :r] * s[:r])
    V2h = Fh[:r, :]
    j2 = woodbury_solve(beta, U2, V2h, v2)
    Cx = Gmh @ C2 @ Gh
    B = Q.T @ Cx
    return dict(x=Gmh @ j2, j2=j2, rank=r, sigma=s, B=B, Bhat=Bhat, Q=Q, beta=beta,
                Ux=Gmh @ U2, Vxh=V2h @ Gh, vx=Gmh @ v2, Gh=Gh, Gmh=Gmh)


# --------------------------------------------------------------------------------------
# Block route (Sec. III-A, IV on an equal-chord mesh): the same filtered operator and
# compressed solution as the projected route, formed from the n x N block
#     B = Q^T (G^-1 S G^-1 N - I/4 - alpha G^-1 D)
# without any N x N product or dense factor, so it reaches the large meshes
# (O(n N^2) work after the assembly).
# --------------------------------------------------------------------------------------


def chord_length(verts) -> float:
    """The common chord h of an equal-chord mesh, as the mean chord.  The vertex coordinates
    of a generated equal-chord mesh are rounded, so its chords agree only to about
    1e-16 |r| / h relative (6e-12 at 16384 vertices on a unit-size curve); spreads up to
    1e-10 are accepted and read as one chord h."""
    h = Mesh(verts).h
    assert np.max(h) - np.min(h) <= 1e-10 * np.mean(h), "mesh is not equal-chord"
    return float(np.mean(h))


def gram_dft_eigs(N: int, h: float):
    """Eigenvalues of the equal-chord Gram matrix G = circ(2h/3; h/6) in DFT order:
    G e_m = lambda_m e_m for e_m = (exp(2 pi i m j / N))_j, lambda_m = h (2 + cos(2 pi m/N)) / 3."""
    return h * (2.0 + np.cos(2.0 * math.pi * np.arange(N) / N)) / 3.0


def gram_power_rows(X, h: float, p: float):
    """X G^p for the rows of X (..., N): G is circulant and symmetric, so G^p is the
    circulant with eigenvalues lambda_m^p and x G^p = ifft(fft(x) lambda^p)."""
    X = np.asarray(X)
    lam = gram_dft_eigs(X.shape[-1], h) ** p
    return np.fft.ifft(np.fft.fft(X, axis=-1) * lam, axis=-1)


def gram_power_cols(X, h: float, p: float):
    """G^p X for the columns of X (N, ...)."""
    return gram_power_rows(np.asarray(X).T, h, p).T


def filtered_block(mats, verts, M: int, alpha: float = 0.0, include_kernel: bool = True):
    """B = Q^T C_x (n x N), C_x = G^-1 S G^-1 N - I/4 - alpha G^-1 D the compact part in
    nodal coordinates, so that the filtered operator (Sec. IV-A) is P C_x = Q B.  The columns
    of Q are eigenvectors of G (Q^T G^-1 = diag(1/g) Q^T), hence
        B = diag(1/g) (Q^T S) G^-1 N - alpha diag(1/g) Q^T D - Q^T / 4."""
    verts = np.asarray(verts)
    N = verts.shape[0]
    h = chord_length(verts)
    Q = fourier_basis(N, M, include_kernel)
    g = gram_eigs(N, h, M, include_kernel)
    Y = gram_power_rows(Q.T @ mats["S"], h, -1.0)             # (Q^T S) G^-1
    B = (Y @ mats["W"]) / g[:, None] - Q.T / 4.0
    if alpha != 0.0:
        B = B - alpha * (Q.T @ mats["D"]) / g[:, None]
    return B, Q, g, h


def compress_block(B, Q, g, h, tol: float):
    """Compression in the paper's orthonormal basis (Sec. IV-C, j2 = G^1/2 x): the filtered
    compact part there is Q B^ with B^ = diag(g^1/2) B G^-1/2.  With the SVD
    B^ = E diag(sigma) F^H and r = #{sigma_i >= tol sigma_1}, the truncation Q E_r E_r^H B^
    reads, back in nodal coordinates, Q B ~= U V^H with
        U = Q diag(g^-1/2) E_r,   V^H = E_r^H diag(g^1/2) B."""
    Bhat = gram_power_rows(np.sqrt(g)[:, None] * B, h, -0.5)
    E, s, _ = np.linalg.svd(Bhat, full_matrices=False)
    r = int(np.sum(s >= tol * s[0])) if tol > 0 else int(np.sum(s > 0))
    U = (Q / np.sqrt(g)[None, :]) @ E[:, :r]
    Vh = E[:, :r].conj().T @ (np.sqrt(g)[:, None] * B)
    return U, Vh, s, r, Bhat


def filtered_condition(beta, Bhat, Q):
    """2-norm condition number of the filtered operator A2 = beta I + Q B^ in the
    orthonormal basis, exactly, from a 2n x 2n matrix.  In an orthonormal basis [Q, Q_perp]
    A2 = [[beta I + B^ Q, B^ Q_perp], [0, beta I]]; with the SVD B^ Q_perp = U_c diag(s_c) V_c^H
    the span of Q_perp V_c carries [[beta I + B^ Q, U_c diag(s_c)], [0, beta I]] and the rest of
    Q_perp (N - 2n dimensions) is mapped to beta times itself."""
    N, n = Q.shape
    if N < 2 * n:
        return float(np.linalg.cond(beta * np.eye(N) + Q @ Bhat))
    C = Bhat - (Bhat @ Q) @ Q.T                                # B^ Q_perp Q_perp^T
    Uc, sc, _ = np.linalg.svd(C, full_matrices=False)
    T = np.zeros((2 * n, 2 * n), dtype=np.complex128)
    T[:n, :n] = beta * np.eye(n) + Bhat @ Q
    T[:n, n:] = Uc * sc[None, :]
    T[n:, n:] = beta * np.eye(n)
    sv = np.linalg.svd(T, compute_uv=False)
    if N > 2 * n:
        sv = np.append(sv, abs(beta))
    return float(np.max(sv) / np.min(sv))


def filtered_solve_blocks(mats, verts, f, M: int, tol: float, alpha: float = 0.0, h2=None,
                          include_kernel: bool = True):
    """The filtered fast direct solver of Sec. IV on an equal-chord mesh, in nodal
    coordinates x (j2 = G^1/2 x):
        v = G^-1 S G^-1 f - alpha G^-1 h2          (right-hand side, Sec. II / IV-A)
        B = Q^T C_x                                (filtered_block)
        U V^H ~= Q B at tol                        (compress_block)
        x = (beta I + U V^H)^-1 v                  (Woodbury, Sec. IV-C)
    Also returns the uncompressed filtered solution x_full = (beta I + Q B)^-1 v (Woodbury
    with the rank-n factors Q, B) and the condition number of the filtered operator."""
    B, Q, g, h = filtered_block(mats, verts, M, alpha, include_kernel)
    beta = (1.0 + 2.0 * alpha) / 4.0
    v = gram_power_cols(mats["S"] @ gram_power_cols(f, h, -1.0), h, -1.0)
    if alpha != 0.0:
        v = v - alpha * gram_power_cols(h2, h, -1.0)
    U, Vh, s, r, Bhat = compress_block(B, Q, g, h, tol)
    x = woodbury_solve(beta, U, Vh, v)
    x_full = woodbury_solve(beta, Q.astype(np.complex128), B, v)
    kappa = filtered_condition(beta, Bhat, Q)
    return dict(x=x, x_full=x_full, rank=r, sigma=s, B=B, U=U, Vh=Vh, vx=v, beta=beta, kappa=kappa, h=h)


# --------------------------------------------------------------------------------------
# Reference solutions and norms
# --------------------------------------------------------------------------------------


def mie_current(k: float, a: float, theta, phi_inc: float, mmax: int | None = None):
    """Exact TE current on a circle of radius a for u_inc = exp(i k d.x):
    j(theta) = -u_tot = -sum_m i^|m| 2 i / (pi k a H_|m|^(1)'(k a)) e^{i m (theta - phi)}."""
    theta = np.asarray(theta, dtype=np.float64)
    if mmax is None:
        mmax = int(k * a + 40)
    ka = k * a
    out = np.zeros(theta.shape, dtype=np.complex128)
    for m in range(-mmax, mmax + 1):
        Hp = special.h1vp(abs(m), ka)
        # e^{i k a cos(t)} = sum_m i^|m| J_|m|(ka) e^{i m t}: the coefficient depends on |m|
        out += -(1j ** abs(m)) * 2j / (math.pi * ka * Hp) * np.exp(1j * m * (theta - phi_inc))
    return out


def circle_spectra(k: float, a: float, m):
    """Continuous eigenvalues on a circle of radius a (Graf addition theorem):
    S: (i pi a/2) J_m H_m ;  N: -(i pi a k^2/2) J_m' H_m' ;  D (principal value):
    (i pi k a/2) J_m H_m' + 1/2."""
    m = np.abs(np.asarray(m))
    ka = k * a
    J = special.jv(m, ka); H = special.hankel1(m, ka)
    Jp = special.jvp(m, ka); Hp = special.h1vp(m, ka)
    s = 0.5j * math.pi * a * J * H
    w = -0.5j * math.pi * a * k * k * Jp * Hp
    d = 0.5j * math.pi * ka * J * Hp + 0.5
    return s, w, d


def g_norm(G, x):
    """||x||_G = sqrt(x^H G x) per column (the L2 norm of the P1 current)."""
    x = np.atleast_2d(x.T).T
    return np.sqrt(np.real(np.einsum("ir,ij,jr->r", np.conj(x), G, x)))


# --------------------------------------------------------------------------------------
# Far field and the adjoint gradient of a far-field misfit (differentiation layer)
# --------------------------------------------------------------------------------------


def farfield_constant(k: float) -> complex:
    """C0 in g(x, y) ~ C0 e^{i k |x|} / sqrt|x| e^{-i k xhat.y} for g = (i/4) H0^(1)(k r)
    (large-argument Hankel form): C0 = (i/4) sqrt(2/(pi k)) e^{-i pi/4} = e^{i pi/4}/sqrt(8 pi k)."""
    return complex(np.exp(0.25j * math.pi) / math.sqrt(8.0 * math.pi * k))


def farfield_matrix(verts, k: float, obs_angles):
    """F (nobs, N) with u_inf(xhat_o) = sum_i F[o, i] x_i for the P1 current x = -u_tot.

    Green's representation of the sound-hard problem (d u_tot/d nu = 0 on the curve):
    u_s(x) = int u_tot(y) d g(x, y)/d nu_y ds_y, and d/d nu_y e^{-i k xhat.y} =
    -i k (xhat.nu_y) e^{-i k xhat.y}, so
        F[o, i] = i k C0 int phi_i(y) (xhat_o.nu_y) e^{-i k xhat_o.y} ds_y,
    which is C0 times the right-hand side f_i of the plane wave travelling along -xhat_o."""
    obs = np.asarray(obs_angles, dtype=np.float64)
    return (farfield_constant(k) * rhs_planewave(verts, k, obs + math.pi)).T


def mie_farfield(k: float, a: float, theta, phi_inc: float, mmax: int | None = None):
    """Exact far field of the sound-hard circle of radius a for u_inc = exp(i k d.x):
    u_s = -sum_m i^|m| J'_|m|(ka)/H'_|m|(ka) H_|m|(k r) e^{i m (theta - phi)} and
    H_m(k r) ~ sqrt(2/(pi k r)) e^{i (k r - m pi/2 - pi/4)} give
    u_inf(theta) = -sqrt(2/(pi k)) e^{-i pi/4} sum_m J'_|m|(ka)/H'_|m|(ka) e^{i m (theta - phi)}."""
    theta = np.asarray(theta, dtype=np.float64)
    if mmax is None:
        mmax = int(k * a + 40)
    ka = k * a
    out = np.zeros(theta.shape, dtype=np.complex128)
    for m in range(-mmax, mmax + 1):
        out += special.jvp(abs(m), ka) / special.h1vp(abs(m), ka) * np.exp(1j * m * (theta - phi_inc))
    return -math.sqrt(2.0 / (math.pi * k)) * np.exp(-0.25j * math.pi) * out


def misfit_blocks(res: dict, F, amplitudes, target):
    """Misfit J(a) = sum_{o,w} |u_ow - t_ow|^2 of the far fields u = F X, X_w = a_w x_w, with
    x = A^-1 v the filtered solution of filtered_solve_blocks (compressed at its tolerance),
    and its gradient in the amplitudes (dJ/dRe a + i dJ/dIm a):
        grad_a_w = 2 (F x_w)^H r_w,   r = u - t."""
    x0 = res["x"]
    a = np.asarray(amplitudes, dtype=np.complex128)
    Fx0 = F @ x0
    u = Fx0 * a[None, :]
    r = u - target
    return dict(J=float(np.sum(np.abs(r) ** 2)), u=u, x0=x0, grad_a=2.0 * np.einsum("ow,ow->w", np.conj(Fx0), r))


def misfit_and_gradients(route: dict, F, amplitudes, target):
    """Misfit J(a, v) = sum_{o,w} |u_ow - t_ow|^2 of the far fields u = F x, x_w = A^-1 (a_w v_w),
    A = beta I + U_x V_x^H the compressed filtered operator of filtered_solve_projected
    (x-coordinates), v_w its preconditioned right-hand sides.

    Gradients in the convention dJ/dRe z + i dJ/dIm z (the one torch uses for complex
    leaves):
        grad_a_w = 2 (F x0_w)^H r_w,  x0_w = A^-1 v_w,  r = u - t;
        grad_v_w = 2 A^-H F^H r_w  (the adjoint solve; a_w folded in: d u_w/d v_w = a_w F A^-1,
                                    so grad_v_w = conj(a_w) 2 A^-H F^H r_w).
    A^-1 and A^-H are dense LU solves of the N x N operator."""
    beta = route["beta"]
    A = beta * np.eye(route["Ux"].shape[0]) + route["Ux"] @ route["Vxh"]
    v = route["vx"]
    a = np.asarray(amplitudes, dtype=np.complex128)
    x0 = np.linalg.solve(A, v)
    u = F @ (x0 * a[None, :])
    r = u - target
    J = float(np.sum(np.abs(r) ** 2))
    Fx0 = F @ x0
    grad_a = 2.0 * np.einsum("ow,ow->w", np.conj(Fx0), r)
    lam = np.linalg.solve(A.conj().T, F.conj().T @ r)
    grad_v = 2.0 * lam * np.conj(a)[None, :]
    return dict(J=J, u=u, x0=x0, grad_a=grad_a, grad_v=grad_v, A=A)
