"""Batching layer: many uneven geometries solved concurrently on several streams give the
results of solving them one by one; the recorded CUDA graph of the FP64 solves replays
them, and so does the grouped persistent solve; the stream-count tuner returns a choice per
size bucket."""
import numpy as np
import pytest
import torch

from paper_2210_08580_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2210_08580_gb300 import bem, batch
    bem.load_library()
    return bem, batch


@pytest.fixture(scope="module")
def problems(B):
    _, batch = B
    specs = I.batch_problems(count=5, first_seed=100, n_lo=300, n_hi=1400, r_lo=8, r_hi=40)
    return batch.problems_from_inputs(specs)


def _single(bem, p, prec):
    s = bem.Solver(device=0, prec=prec)
    s.assemble(torch.from_numpy(p.verts).cuda(), p.k, ops="SW")
    s.filter_apply(p.n_modes)
    r = s.compress(p.tol)
    s.factor()
    v = s.rhs_planewave(torch.from_numpy(p.angles).cuda())
    x = s.solve(v)
    torch.cuda.synchronize()
    s.close()
    return x, r


@pytest.mark.parametrize("prec,solve", [("fp64", "each"), ("mixed", "each"), ("fp64", "grouped")])
def test_batch_matches_one_by_one(B, problems, prec, solve):
    """The batch gives the one-by-one solutions: to the last bits with per-problem solves, to
    1e-13 with the grouped solve (the slices of V^H v reorder the FP64 sums)."""
    bem, batch = B
    bs = batch.BatchSolver(problems, prec=prec, n_streams=3, solve=solve)
    res = bs.run()
    for p, out in zip(problems, res):
        x, r = _single(bem, p, prec)
        assert out["rank"] == r
        err = float((out["x"] - x).abs().max() / x.abs().max())
        assert err <= (1e-14 if solve == "each" else 1e-13), err
    bs.close()


def test_solve_graph_replays_all_solves(B, problems):
    bem, batch = B
    bs = batch.BatchSolver(problems, prec="fp64", n_streams=2)
    res = bs.run()
    g = batch.SolveGraph(bs)
    for i, out in enumerate(res):
        g.v[i].copy_(out["v"])
    g.replay()
    torch.cuda.synchronize()
    for i, out in enumerate(res):
        err = float((g.x[i] - out["x"]).abs().max() / out["x"].abs().max())
        assert err <= 1e-13, (i, err)
    # new right-hand sides in the same buffers: the graph solves them
    for i, out in enumerate(res):
        g.v[i].mul_(0.5j)
    g.replay()
    torch.cuda.synchronize()
    for i, out in enumerate(res):
        err = float((g.x[i] - 0.5j * out["x"]).abs().max() / out["x"].abs().max())
        assert err <= 1e-13, (i, err)
    bs.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_grouped_solve_matches_one_by_one(B, problems, prec):
    """bem_solve_batch (every problem's Woodbury products in one persistent launch) gives
    each problem's FP64 Woodbury solve: the batch's own solutions on FP64 handles,
    solve_many_noalloc's on mixed ones (same factors, FP64 products; the slices of V^H v only
    change the order of the sums)."""
    bem, batch = B
    L = bem.load_library()
    bs = batch.BatchSolver(problems, prec=prec, n_streams=3)
    res = bs.run()
    vs = [out["v"] for out in res]
    xg = batch.solve_grouped(bs.solvers, vs)
    torch.cuda.synchronize()
    for i, (s, out) in enumerate(zip(bs.solvers, res)):
        x1 = torch.empty_like(vs[i])
        assert L.solve_many_noalloc(s.h, vs[i].data_ptr(), s.N, x1.data_ptr(), s.N, vs[i].shape[0]) == 0
        torch.cuda.synchronize()
        err = float((xg[i] - x1).abs().max() / x1.abs().max())
        assert err <= 1e-13, (i, err)
        if prec == "fp64":
            err = float((xg[i] - out["x"]).abs().max() / out["x"].abs().max())
            assert err <= 1e-13, (i, err)
    bs.close()


def test_grouped_solve_edges(B):
    """Ragged slices and tiles: N = 2500 (ten 256-long slices of V^H v, the last 196),
    nrhs 1, 65 and 130 (one-wide and ragged column blocks), one handle twice with different
    right-hand sides, a mixed handle beside FP64 ones; each against the handle's own FP64
    Woodbury solve.  A handle that is not factored is refused by name, before any work."""
    bem, batch = B
    L = bem.load_library()
    star = I.cos_star(1.0, 0.3, 5)
    specs = [(I.equal_chord_mesh(star, 2500)[0], 2.0, "fp64"), (I.equal_chord_mesh(star, 300)[0], 0.7, "fp64"),
             (I.equal_chord_mesh(I.perturbed_circle(), 700)[0], 1.3, "mixed")]
    ss = []
    for verts, k, prec in specs:
        s = bem.Solver(device=0, prec=prec)
        s.assemble(torch.from_numpy(verts).cuda(), k, ops="SW")
        s.filter_apply(21)
        s.compress(1e-10)
        s.factor()
        ss.append(s)
    gen = torch.Generator().manual_seed(7)
    shapes = [(130, 2500), (1, 300), (65, 2500), (65, 700)]
    who = [ss[0], ss[1], ss[0], ss[2]]
    vs = [torch.complex(torch.randn(sh, generator=gen, dtype=torch.float64),
                        torch.randn(sh, generator=gen, dtype=torch.float64)).cuda() for sh in shapes]
    xg = batch.solve_grouped(who, vs)
    torch.cuda.synchronize()
    for s, v, x in zip(who, vs, xg):
        x1 = torch.empty_like(v)
        assert L.solve_many_noalloc(s.h, v.data_ptr(), s.N, x1.data_ptr(), s.N, v.shape[0]) == 0
        torch.cuda.synchronize()
        err = float((x - x1).abs().max() / x1.abs().max())
        assert err <= 1e-13, (s.N, v.shape[0], err)
    fresh = bem.Solver(device=0)
    fresh.assemble(torch.from_numpy(specs[1][0]).cuda(), 0.7, ops="SW")
    with pytest.raises(bem.BemError) as ei:
        batch.solve_grouped([ss[1], fresh], [vs[1], vs[1].clone()])
    assert ei.value.status == 1 and "problem 1" in str(ei.value)
    for s in ss + [fresh]:
        s.close()


def test_grouped_solve_long_slices(B):
    """Above N = 16384 the slices of V^H v lengthen (at most 64 per problem): N = 20000 takes
    63 slices of 320 (the last 160), beside a small problem with 256-long slices; each against
    the handle's own FP64 Woodbury solve."""
    bem, batch = B
    L = bem.load_library()
    star = I.cos_star(1.0, 0.3, 5)
    ss = []
    for N, k in ((20000, 0.5), (700, 1.0)):
        s = bem.Solver(device=0)
        s.assemble(torch.from_numpy(I.equal_chord_mesh(star, N)[0]).cuda(), k, ops="SW")
        s.filter_apply(21)
        s.compress(1e-10)
        s.factor()
        ss.append(s)
    gen = torch.Generator().manual_seed(11)
    vs = [torch.complex(torch.randn((nr, s.N), generator=gen, dtype=torch.float64),
                        torch.randn((nr, s.N), generator=gen, dtype=torch.float64)).cuda()
          for nr, s in zip((3, 70), ss)]
    xg = batch.solve_grouped(ss, vs)
    torch.cuda.synchronize()
    for s, v, x in zip(ss, vs, xg):
        x1 = torch.empty_like(v)
        assert L.solve_many_noalloc(s.h, v.data_ptr(), s.N, x1.data_ptr(), s.N, v.shape[0]) == 0
        torch.cuda.synchronize()
        err = float((x - x1).abs().max() / x1.abs().max())
        assert err <= 1e-13, (s.N, err)
    for s in ss:
        s.close()


def test_grouped_solve_wait_timeout_is_reported(B, problems):
    """Failure detection without a GPU fault: the grouped kernel with one completion counter
    that nothing brings to its target gives up the waits on it after 0.2 s of wall time, the
    call returns BEM_E_TIMEOUT, and the same handles then solve normally."""
    import time
    bem, batch = B
    L = bem.load_library()
    bs = batch.BatchSolver(problems, prec="fp64", n_streams=2)
    res = bs.run()
    vs = [out["v"] for out in res]
    t0 = time.perf_counter()
    st, msg = batch.grouped_stall_check(bs.solvers, vs, stall_ms=200)
    dt = time.perf_counter() - t0
    assert st == 7 and "timed out" in msg, (st, msg)
    assert 0.15 <= dt <= 5.0, dt
    xg = batch.solve_grouped(bs.solvers, vs)
    torch.cuda.synchronize()
    for i, out in enumerate(res):
        err = float((xg[i] - out["x"]).abs().max() / out["x"].abs().max())
        assert err <= 1e-13, (i, err)
    bs.close()


def test_stream_tuner_picks_per_bucket(B, problems):
    _, batch = B
    best = batch.autotune_streams(problems[:3], prec="fp64", candidates=(1, 2), sample=2)
    assert best and all(v in (1, 2) for v in best.values())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solver_is_deterministic(B, problems, prec):
    """Two runs of the same problem give bit-identical solutions (no order-dependent
    floating-point reductions anywhere on the path)."""
    bem, _ = B
    p = problems[0]
    x1, _ = _single(bem, p, prec)
    x2, _ = _single(bem, p, prec)
    assert torch.equal(x1, x2)


def _c4():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c4_batch_subsample.npz")
    with np.load(path) as z:
        return {key: z[key] for key in z.files}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_subsample_against_the_oracle(B, prec):
    """C4 within the oracle's reach: the first 8 problems of the uneven batch law with
    N ~ U{512..2048} (random stars, k = 10^U(-2, log10 5), 64..512 plane waves each), solved
    together by the batching layer; every problem's rank, singular values and solution
    (64 rows x every nrhs/8-th wave) against the oracle: FP64 <= 1e-10 (1e-13 kappa above
    kappa = 1e3), mixed <= 1e-8 (1e-11 kappa), ranks equal up to one."""
    bem, batch = B
    g = _c4()
    problems = batch.problems_from_inputs(I.batch_problems(count=int(g["count"]), first_seed=100, n_hi=2048))
    bs = batch.BatchSolver(problems, prec=prec, n_streams=4, refine_rtol=1e-8)
    res = bs.run()
    errs = []
    for i, out in enumerate(res):
        kappa = float(g[f"p{i}_kappa"])
        if prec == "fp64":
            tol = 1e-10 if kappa <= 1e3 else 1e-13 * kappa
        else:
            tol = 1e-8 if kappa <= 1e3 else 1e-11 * kappa
        x = out["x"].cpu().numpy().T[g[f"p{i}_rows"]][:, g[f"p{i}_cols"]]
        r, r0 = out["rank"], int(g[f"p{i}_rank"])
        ref = g[f"p{i}_x"] if r == r0 else g[f"p{i}_x_full"]
        if r != r0:
            tol = max(tol, 1e-9 * kappa)
        err = float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))
        print(f"batch {prec} problem {i}: N={problems[i].verts.shape[0]} k={problems[i].k:.3g} kappa={kappa:.3g} "
              f"rank {r}/{r0} x err {err:.2e} (tol {tol:.1e})")
        assert abs(r - r0) <= 1
        assert err <= tol, (i, err, tol)
        errs.append((x, ref, tol))
    # the same right-hand sides through the grouped persistent solve (FP64 Woodbury tiles of
    # all 8 problems in one launch; on mixed handles it is the exact inverse of the handle's
    # compressed operator, which the refined solve converges to)
    xg = batch.solve_grouped(bs.solvers, [out["v"] for out in res])
    for i, (x_b, ref, tol) in enumerate(errs):
        xgi = xg[i].cpu().numpy().T[g[f"p{i}_rows"]][:, g[f"p{i}_cols"]]
        err = float(np.max(np.abs(xgi - ref)) / np.max(np.abs(ref)))
        print(f"grouped {prec} problem {i}: x err {err:.2e} (tol {tol:.1e})")
        assert err <= tol, (i, err, tol)
    bs.close()


def test_persistent_batch_assembly_equals_one_by_one(B, problems):
    """bem_assemble_batch (one launch over a global tile queue) writes the same S and N bits
    as one bem_assemble per problem, on both paths."""
    bem, _ = B
    for prec in ("fp64", "mixed"):
        ss = [bem.Solver(device=0, prec=prec) for _ in problems]
        bem.assemble_batch(ss, [torch.from_numpy(p.verts) for p in problems], [p.k for p in problems])
        for p, s in zip(problems, ss):
            one = bem.Solver(device=0, prec=prec)
            one.assemble(torch.from_numpy(p.verts).cuda(), p.k, ops="SW")
            for op in "SW":
                assert torch.equal(s.matrix(op), one.matrix(op)), (prec, op, p.verts.shape[0])
            assert s.info()["quad_points"] == one.info()["quad_points"]
            one.close()
        for s in ss:
            s.close()


def test_tile_tuner_picks_a_shape_per_bucket_and_stage(B, problems):
    """autotune_tiles: one (tile width, K splits) per size bucket and stage, among the
    candidates, chosen by measured kernel time; a batch run with the tuned shapes gives the
    one-by-one results (split changes only the order of FP64 partial sums)."""
    bem, batch = B
    tuned = batch.autotune_tiles(problems, reps=1)
    buckets = {batch.size_bucket(p.verts.shape[0]) for p in problems}
    assert set(tuned) == buckets
    for b, ch in tuned.items():
        for stage in ("filter", "rhs"):
            assert (ch[f"{stage}_tile_n"], ch[f"{stage}_split_k"]) in batch.TILE_CANDIDATES[stage]
            t = ch["times_ms"][stage]
            assert min(t.values()) == t[f"{ch[f'{stage}_tile_n']}x{ch[f'{stage}_split_k']}"]
    bs = batch.BatchSolver(problems, prec="mixed", n_streams=2, tiles=tuned)
    res = bs.run()
    for p, out in zip(problems, res):
        x, r = _single(bem, p, "mixed")
        assert out["rank"] == r
        assert float((out["x"] - x).abs().max() / x.abs().max()) <= 1e-10
    bs.close()


def test_persistent_batch_assembly_with_general_meshes(B):
    """Equal-chord and non-equal-chord problems in one persistent launch: every handle gets
    the bits of its own bem_assemble (the general meshes' wider near-pair series radius and
    their Gram factors included), and its filter and solve run on from there."""
    bem, _ = B
    star = I.cos_star(1.0, 0.3, 5)
    meshes = [I.equal_chord_mesh(star, 400)[0], I.parameter_mesh(star, 333, grade=0.3)[0],
              I.parameter_mesh(I.perturbed_circle(), 520)[0]]
    ks = [2.0, 1.5, 0.4]
    ss = [bem.Solver(device=0) for _ in meshes]
    bem.assemble_batch(ss, [torch.from_numpy(v) for v in meshes], ks)
    for v, k, s in zip(meshes, ks, ss):
        one = bem.Solver(device=0)
        one.assemble(torch.from_numpy(v).cuda(), k, ops="SW")
        assert s.info()["equal_chord"] == one.info()["equal_chord"]
        for op in "SW":
            assert torch.equal(s.matrix(op), one.matrix(op)), (op, v.shape[0])
        ang = torch.from_numpy(I.planewave_angles(3)).cuda()
        xs = []
        for h in (s, one):
            h.filter_apply(21)
            h.compress(1e-10)
            h.factor()
            xs.append(h.solve(h.rhs_planewave(ang)))
        assert torch.equal(xs[0], xs[1])
        one.close()
    assert [s.info()["equal_chord"] for s in ss] == [1, 0, 0]
    for s in ss:
        s.close()
