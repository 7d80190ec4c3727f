"""The paper's own workloads (Sec. V), on the GPU path, with the line ("dipole") source:

* Table I: perturbed circle r = 2 + 0.2 sin 8t, compression tolerance 1e-3, filtering point
  200 (n = 201 modes), N = 1004 .. 8032;
* Fig. 3: ellipse with semi-axes 1.42 and 1.32 at k = 0.4, tolerance 6e-6, filtering point 21,
  error and rank against the refinement.

The paper prints neither the wavenumber nor the source position of Table I; they are read as
k = 0.4 (the ellipse's) and a line source at r0 = (3, 0).  Its printed values are therefore
checked as bands (rank of order 24 that stops growing with N, the compressed solution within
the tolerance of the uncompressed one, skeleton memory growing linearly), not digit by digit,
while the GPU results are checked against the CPU oracle on the smallest mesh of each sweep.
"""
import math
import os

import numpy as np
import pytest
import torch

from oracle import bem_oracle as O
from paper_2210_08580_gb300 import inputs as I

pytestmark = pytest.mark.gpu

K_PAPER = 0.4
SOURCE = np.array([[3.0, 0.0]])
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def B():
    from paper_2210_08580_gb300 import bem
    bem.load_library()
    return bem


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _g_norm(x, h):
    """||x||_G per column of x (nsrc, N) for the equal-chord Gram matrix circ(2h/3; h/6)."""
    Gx = (h / 6.0) * (torch.roll(x, 1, dims=1) + 4.0 * x + torch.roll(x, -1, dims=1))
    return torch.sqrt((x.conj() * Gx).real.sum(dim=1))


def _compressed_and_full(B, verts, k, M, tol, src=SOURCE, prec="fp64"):
    """GPU path: line-source RHS, solutions of the compressed (tol) and the uncompressed
    (tol = 0: every filtered mode kept) filtered operator; rank and G-norm error."""
    s = B.Solver(device=0, prec=prec)
    s.assemble(_cuda(verts), k, ops="SW")
    v = s.rhs_pointsource(_cuda(src))
    s.filter_apply(2 * M + 1)
    s.compress(0.0)
    s.factor()
    x_full = s.solve(v)
    r = s.compress(tol)
    s.factor()
    x = s.solve(v)
    h = s.info()["h"]
    err = float((_g_norm(x - x_full, h) / _g_norm(x_full, h)).max())
    s.close()
    return dict(x=x, x_full=x_full, rank=r, err=err, h=h)


def test_pointsource_rhs_matches_oracle(B):
    v, _, _ = I.equal_chord_mesh(I.cos_star(1.0, 0.3, 5), 301)
    k = 2.0
    src = np.array([[3.0, 0.0], [-2.5, 1.0], [0.2, -1.9]])
    s = B.Solver(device=0)
    s.assemble(_cuda(v), k, ops="SWD")
    f, vv = s.rhs_pointsource(_cuda(src), want_f=True)
    f_o = O.rhs_pointsource(v, k, src)
    assert float(np.max(np.abs(f.cpu().numpy().T - f_o)) / np.max(np.abs(f_o))) <= 1e-13
    mats = O.assemble(v, k, "SWD")
    ref = O.filtered_solve_blocks(mats, v, f_o, 20, 1e-10)
    assert float(np.max(np.abs(vv.cpu().numpy().T - ref["vx"])) / np.max(np.abs(ref["vx"]))) <= 1e-12
    # the CFIE right-hand side adds -alpha G^-1 h2 with h2 = <phi, u_inc>
    s.filter_apply(41, alpha=0.5)
    vc = s.rhs_pointsource(_cuda(src))
    refc = O.filtered_solve_blocks(mats, v, f_o, 20, 1e-10, alpha=0.5, h2=O.rhs_pointsource_h(v, k, src))
    assert float(np.max(np.abs(vc.cpu().numpy().T - refc["vx"])) / np.max(np.abs(refc["vx"]))) <= 1e-12
    s.compress(1e-10)
    s.factor()
    x = s.solve(vc).cpu().numpy().T
    assert float(np.max(np.abs(x - refc["x"])) / np.max(np.abs(refc["x"]))) <= 1e-10
    s.close()


def _table1():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "table1.txt")) if ln.strip() and ln[0] != "#"]
    return {int(r[0]): dict(err=float(r[1]), dense_mb=float(r[2]), skel_mb=float(r[3])) for r in rows}


def test_table1_perturbed_circle(B):
    """Table I (Sec. V): perturbed circle, tol 1e-3, filtering point 200, N = 1004 .. 8032."""
    table = _table1()
    M, tol = 100, 1e-3
    res = {}
    for N in sorted(table):
        verts, _, _ = I.equal_chord_mesh(I.perturbed_circle(), N)
        res[N] = _compressed_and_full(B, verts, K_PAPER, M, tol)
        skel_mb = 2 * N * res[N]["rank"] * 16 / 1e6                 # U and V, complex128
        dense_mb = 16 * N * N / 1e6
        print(f"Table I N={N}: rank {res[N]['rank']}, error {res[N]['err']:.2e} (paper {table[N]['err']:.2e}), "
              f"skeleton {skel_mb:.2f} MB (paper {table[N]['skel_mb']}), dense {dense_mb:.0f} MB "
              f"(paper {table[N]['dense_mb']:.0f} MB)")
        # the dense column is 16 N^2 bytes (complex128), in MB of 10^6 bytes
        assert abs(dense_mb - table[N]["dense_mb"]) <= 0.6
        # the compressed solution stays within the tolerance of the uncompressed one, at the
        # level the paper prints (0.23e-3 .. 0.24e-3; within a factor of two under the k and
        # source readings)
        assert res[N]["err"] <= tol, (N, res[N]["err"])
        assert 0.5 * table[N]["err"] <= res[N]["err"] <= 2.0 * table[N]["err"], (N, res[N]["err"])
        res[N]["skel_mb"] = skel_mb
    ranks = [res[N]["rank"] for N in sorted(res)]
    # the rank is of the paper's order (24 from N = 2008 on) and stops growing with the
    # refinement, so the skeleton's memory grows linearly in N
    assert all(8 <= r <= 80 for r in ranks), ranks
    assert max(ranks[1:]) - min(ranks[1:]) <= 2, ranks
    per_n = [res[N]["skel_mb"] / N for N in sorted(res)[1:]]
    assert max(per_n) <= 1.15 * min(per_n), per_n
    # the smallest mesh against the CPU oracle (rank, uncompressed and compressed solutions)
    N0 = min(table)
    verts, _, _ = I.equal_chord_mesh(I.perturbed_circle(), N0)
    mats = O.assemble(verts, K_PAPER, "SW", workers=min(16, os.cpu_count() or 1))
    ref = O.filtered_solve_blocks(mats, verts, O.rhs_pointsource(verts, K_PAPER, SOURCE), M, tol)
    xg = res[N0]["x_full"].cpu().numpy().T
    e_full = float(np.max(np.abs(xg - ref["x_full"])) / np.max(np.abs(ref["x_full"])))
    assert e_full <= 1e-13 * max(1e3, ref["kappa"]), (e_full, ref["kappa"])
    assert abs(res[N0]["rank"] - ref["rank"]) <= 1
    if res[N0]["rank"] == ref["rank"]:
        xc = res[N0]["x"].cpu().numpy().T
        assert float(np.max(np.abs(xc - ref["x"])) / np.max(np.abs(ref["x"]))) <= 1e-10


def test_fig3_ellipse_error_and_rank_against_refinement(B):
    """Fig. 3 (Sec. V): ellipse 1.42 x 1.32, k = 0.4, tol 6e-6, filtering point 21 (M = 10):
    with refinement the error against the uncompressed operator stays at the tolerance's
    level and the rank saturates to a constant."""
    M, tol = 10, 6e-6
    Ns = (64, 128, 256, 512, 1024, 2048, 4096)
    res = {}
    for N in Ns:
        verts, _, _ = I.equal_chord_mesh(I.ellipse(1.42, 1.32), N)
        res[N] = _compressed_and_full(B, verts, K_PAPER, M, tol)
        print(f"Fig. 3 N={N} 1/h={1 / res[N]['h']:.1f}: rank {res[N]['rank']}, error {res[N]['err']:.2e}")
        assert res[N]["err"] <= 10 * tol, (N, res[N]["err"])
        assert res[N]["rank"] <= 2 * M + 1
    ranks = [res[N]["rank"] for N in Ns]
    assert max(ranks[-3:]) - min(ranks[-3:]) <= 1, ranks
    # smallest mesh against the oracle
    verts, _, _ = I.equal_chord_mesh(I.ellipse(1.42, 1.32), Ns[0])
    mats = O.assemble(verts, K_PAPER, "SW")
    ref = O.filtered_solve_blocks(mats, verts, O.rhs_pointsource(verts, K_PAPER, SOURCE), M, tol)
    assert abs(res[Ns[0]]["rank"] - ref["rank"]) <= 1
    xg = res[Ns[0]]["x_full"].cpu().numpy().T
    assert float(np.max(np.abs(xg - ref["x_full"])) / np.max(np.abs(ref["x_full"]))) <= 1e-10


def _g_norm_mesh(x, verts):
    """||x||_G per row of x (nsrc, N) for the P1 Gram matrix of the polygon verts, any chords:
    (G x)_i = (h_{i-1} + h_i)/3 x_i + h_{i-1}/6 x_{i-1} + h_i/6 x_{i+1}."""
    v = torch.from_numpy(verts).to(x.device)
    h = torch.linalg.norm(torch.roll(v, -1, 0) - v, dim=1)
    hp = torch.roll(h, 1)
    Gx = (hp + h) / 3 * x + hp / 6 * torch.roll(x, 1, dims=1) + h / 6 * torch.roll(x, -1, dims=1)
    return torch.sqrt((x.conj() * Gx).real.sum(dim=1))


def test_table1_on_polar_uniform_meshes(B):
    """Table I (Sec. V) on meshes uniform in the polar angle, whose chords follow the curve's
    speed (1.43x apart): a non-homogeneous discretisation, filtered through the computed
    lowest eigenvectors of L~ (Sec. III-A).  The compressed solution stays within the paper's
    printed error band of the uncompressed one at every N, the rank stops growing from
    N = 2008 on, the skeleton grows linearly (the oracle's literal route gives rank 31 and 15,
    error 2.23e-4, at N = 1004 and 2008)."""
    table = _table1()
    M, tol = 100, 1e-3
    res = {}
    for N in sorted(table):
        verts, _ = I.parameter_mesh(I.perturbed_circle(), N)
        s = B.Solver(device=0)
        s.assemble(_cuda(verts), K_PAPER, ops="SW")
        assert s.info()["equal_chord"] == 0
        v = s.rhs_pointsource(_cuda(SOURCE))
        s.filter_apply(2 * M + 1)
        s.compress(0.0)
        s.factor()
        x_full = s.solve(v)
        r = s.compress(tol)
        s.factor()
        x = s.solve(v)
        err = float((_g_norm_mesh(x - x_full, verts) / _g_norm_mesh(x_full, verts)).max())
        s.close()
        res[N] = dict(rank=r, err=err, skel_mb=2 * N * r * 16 / 1e6)
        print(f"Table I, polar-uniform mesh, N={N}: rank {r}, error {err:.2e} (paper {table[N]['err']:.2e}), "
              f"skeleton {res[N]['skel_mb']:.2f} MB (paper {table[N]['skel_mb']})")
        assert err <= tol, (N, err)
        assert 0.5 * table[N]["err"] <= err <= 2.0 * table[N]["err"], (N, err)
    ranks = [res[N]["rank"] for N in sorted(res)]
    assert all(8 <= r <= 80 for r in ranks), ranks
    assert max(ranks[1:]) - min(ranks[1:]) <= 2, ranks
    per_n = [res[N]["skel_mb"] / N for N in sorted(res)[1:]]
    assert max(per_n) <= 1.15 * min(per_n), per_n


def test_fig3_ellipse_on_polar_uniform_meshes(B):
    """Fig. 3 (Sec. V) on ellipse meshes uniform in the polar angle (non-equal chords): the
    compressed solution stays at the tolerance's level of the uncompressed one and the rank
    saturates with refinement; the smallest mesh against the oracle's literal route."""
    M, tol = 10, 6e-6
    Ns = (64, 128, 256, 512, 1024, 2048, 4096)
    res = {}
    for N in Ns:
        verts, _ = I.parameter_mesh(I.ellipse(1.42, 1.32), N)
        s = B.Solver(device=0)
        s.assemble(_cuda(verts), K_PAPER, ops="SW")
        assert s.info()["equal_chord"] == 0
        v = s.rhs_pointsource(_cuda(SOURCE))
        s.filter_apply(2 * M + 1)
        s.compress(0.0)
        s.factor()
        x_full = s.solve(v)
        r = s.compress(tol)
        s.factor()
        x = s.solve(v)
        err = float((_g_norm_mesh(x - x_full, verts) / _g_norm_mesh(x_full, verts)).max())
        s.close()
        res[N] = dict(rank=r, err=err, x_full=x_full)
        print(f"Fig. 3, polar-uniform mesh, N={N}: rank {r}, error {err:.2e}")
        assert err <= 10 * tol, (N, err)
        assert r <= 2 * M + 1
    ranks = [res[N]["rank"] for N in Ns]
    assert max(ranks[-3:]) - min(ranks[-3:]) <= 1, ranks
    verts, _ = I.parameter_mesh(I.ellipse(1.42, 1.32), Ns[0])
    mats = O.assemble(verts, K_PAPER, "SW")
    ref = O.filtered_solve_literal(mats, verts, O.rhs_pointsource(verts, K_PAPER, SOURCE), 2 * M + 1, tol)
    assert abs(res[Ns[0]]["rank"] - ref["rank"]) <= 1
    xg = res[Ns[0]]["x_full"].cpu().numpy().T
    assert float(np.max(np.abs(xg - ref["x_full"])) / np.max(np.abs(ref["x_full"]))) <= 1e-10
