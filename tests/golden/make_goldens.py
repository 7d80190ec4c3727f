#!/usr/bin/env python
"""Writes the stored oracle results that the full-size GPU parity tests compare against.

Calls only the CPU oracle (``oracle/bem_oracle.py``, block route of Sec. III-A / IV) and the
seeded input generators; nothing here touches the CUDA path.  For each configuration it
stores, in ``tests/golden/<name>.npz``:

  rows            256 sampled vertex indices (seeded)
  angles          the 16 plane-wave angles solved (every nrhs/16-th of the configuration's
                  nrhs uniform angles, phi_w = 2 pi w / nrhs)
  x, x_full       compressed and uncompressed filtered solutions at ``rows`` (16 columns)
  vx              preconditioned right-hand side G^-1 S G^-1 f at ``rows``
  xnorm_G         G-norm of each full solution column
  sigma, rank     singular values of the filtered compact part, rank at the tolerance
  kappa           condition number of the filtered operator (orthonormal basis)
  c_rowsum        max_i sum_j |N_ij| / |sum_j N_ij|: how much the rounding of N's entries to
                  FP64 (relative 2^-53 each) can move the row sums N 1, which at low k are
                  O(k^2) of the entries and carry the constant mode's eigenvalue

and a summary with the oracle's wall time per phase and the host's core count in
``tests/golden/oracle_runs.json``.

Configurations: star r = 1 + 0.3 cos 5t, N = 4096, k in {1e-3, 1e-2, 1e-1, 1, 5}, n = 201,
tol 1e-10 (256 plane waves); random 8-harmonic star of seed 0, N = 16384, k = 2, n = 201,
tol 1e-10 (1024 plane waves); a subsample of the uneven batch (run_c4); for the
differentiation layer, the C5 misfit (run_c5); and a non-equal-chord mesh (run_general: the
Table I curve meshed uniformly in the polar angle at the paper's N = 2008, by the literal route).

    python tests/golden/make_goldens.py [--workers W] [--only c2|c3|c4|c5|general]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

C2_KS = (1e-3, 1e-2, 1e-1, 1.0, 5.0)


def configs():
    from paper_2210_08580_gb300 import inputs as I
    out = []
    for k in C2_KS:
        out.append(dict(name=f"c2_star_n4096_k{k:g}", curve=I.cos_star(1.0, 0.3, 5), N=4096, k=k, M=100,
                        tol=1e-10, nrhs=256))
    out.append(dict(name="c3_random_star0_n16384", curve=I.random_star(0), N=16384, k=2.0, M=100, tol=1e-10,
                    nrhs=1024))
    return out


def run(cfg, workers):
    from oracle import bem_oracle as O
    from paper_2210_08580_gb300 import inputs as I
    N = cfg["N"]
    verts, _, _ = I.equal_chord_mesh(cfg["curve"], N)
    w = np.arange(0, cfg["nrhs"], cfg["nrhs"] // 16)
    angles = I.planewave_angles(cfg["nrhs"])[w]
    rows = np.sort(np.random.default_rng(12345).choice(N, 256, replace=False))
    t = {}
    t0 = time.perf_counter()
    mats = O.assemble(verts, cfg["k"], "SW", workers=workers)
    t["assemble"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    f = O.rhs_planewave(verts, cfg["k"], angles)
    t["rhs_16"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    res = O.filtered_solve_blocks(mats, verts, f, cfg["M"], cfg["tol"])
    t["block_route"] = time.perf_counter() - t0
    G_norm = np.sqrt(np.real(np.sum(np.conj(res["x"]) * O.gram_power_cols(res["x"], res["h"], 1.0), axis=0)))
    c_rowsum = float(np.max(np.abs(mats["W"]).sum(axis=1) / np.abs(mats["W"].sum(axis=1))))
    np.savez(os.path.join(HERE, cfg["name"] + ".npz"), rows=rows, angles=angles, x=res["x"][rows],
             x_full=res["x_full"][rows], vx=res["vx"][rows], xnorm_G=G_norm, sigma=res["sigma"],
             rank=np.int64(res["rank"]), kappa=np.float64(res["kappa"]), c_rowsum=np.float64(c_rowsum),
             N=np.int64(N), k=np.float64(cfg["k"]),
             M=np.int64(cfg["M"]), tol=np.float64(cfg["tol"]))
    xr = res["x"]
    comp_err = float(np.max(np.abs(xr - res["x_full"])) / np.max(np.abs(res["x_full"])))
    return dict(name=cfg["name"], N=N, k=cfg["k"], n=2 * cfg["M"] + 1, tol=cfg["tol"], rank=res["rank"],
                kappa=res["kappa"], c_rowsum=c_rowsum, compressed_vs_uncompressed=comp_err, seconds=t)


C5_N, C5_K, C5_M, C5_NRHS, C5_NOBS = 8192, 1.0, 100, 128, 360
C5_COEFS = (0, 3, 8, 13)          # cos 1, cos 4, sin 1, sin 6: the coefficients differenced
C5_H = 1e-6


def c5_curve(coef):
    from paper_2210_08580_gb300 import inputs as I
    m = len(coef) // 2
    return I.PolarCurve(r0=1.0, cos_coef=tuple(coef[:m]), sin_coef=tuple(coef[m:]))


def c5_misfit(coef, target, workers):
    """J, grad_a and the far fields of the C5 star with coefficients coef (unit amplitudes)."""
    from oracle import bem_oracle as O
    from paper_2210_08580_gb300 import inputs as I
    verts, _, _ = I.equal_chord_mesh(c5_curve(coef), C5_N)
    ang = I.planewave_angles(C5_NRHS)
    obs = 2.0 * np.pi * np.arange(C5_NOBS) / C5_NOBS
    mats = O.assemble(verts, C5_K, "SW", workers=workers)
    res = O.filtered_solve_blocks(mats, verts, O.rhs_planewave(verts, C5_K, ang), C5_M, 0.0)
    F = O.farfield_matrix(verts, C5_K, obs)
    if target is None:
        return F @ res["x"]
    return O.misfit_blocks(res, F, np.ones(C5_NRHS), target)


def run_c5(workers):
    """C5 (differentiation): random Fourier star of seed 200 (16 coefficients), N = 8192, k = 1,
    n = 201 (no truncation), 128 plane waves, 360 observation angles; target = the far field of
    the seed-201 star.  Stores the target, the misfit and its amplitude gradient at unit
    amplitudes, and central differences (h = 1e-6) of the misfit in 4 coefficients."""
    from paper_2210_08580_gb300 import inputs as I
    t0 = time.perf_counter()
    c0 = np.concatenate(I.fourier_star_seeded(200))
    target = c5_misfit(np.concatenate(I.fourier_star_seeded(201)), None, workers)
    base = c5_misfit(c0, target, workers)
    fd = []
    for p in C5_COEFS:
        e = np.zeros_like(c0)
        e[p] = C5_H
        fd.append((c5_misfit(c0 + e, target, workers)["J"] - c5_misfit(c0 - e, target, workers)["J"]) / (2 * C5_H))
    np.savez(os.path.join(HERE, "c5_fourier_star200_n8192.npz"), coef=c0, target=target, J=np.float64(base["J"]),
             grad_a=base["grad_a"], coefs_fd=np.array(C5_COEFS), fd=np.array(fd), h=np.float64(C5_H),
             N=np.int64(C5_N), k=np.float64(C5_K), M=np.int64(C5_M))
    return dict(name="c5_fourier_star200_n8192", N=C5_N, k=C5_K, J=base["J"], fd=fd,
                seconds={"total": time.perf_counter() - t0})


C4_COUNT, C4_NHI = 8, 2048


def run_c4(workers):
    """C4 subsample within the oracle's reach: the first 8 problems of the uneven batch law
    (random stars of seeds 100.., k = 10^U(-2, log10 5), 64..512 plane waves) with
    N ~ U{512..2048}; n = min(201, 2 floor(N/8) + 1), tol 1e-10.  Per problem: the solution
    at 64 seeded rows for every (nrhs // 8)-th plane wave, sigma, rank, kappa."""
    from oracle import bem_oracle as O
    from paper_2210_08580_gb300 import inputs as I
    t0 = time.perf_counter()
    out = {}
    for i, spec in enumerate(I.batch_problems(count=C4_COUNT, first_seed=100, n_hi=C4_NHI)):
        verts, _, _ = I.equal_chord_mesh(spec.curve, spec.N)
        M = min(201, 2 * (spec.N // 8) + 1) // 2
        w = np.arange(0, spec.nrhs, spec.nrhs // 8)
        angles = I.planewave_angles(spec.nrhs)[w]
        rows = np.sort(np.random.default_rng(777 + i).choice(spec.N, 64, replace=False))
        mats = O.assemble(verts, spec.k, "SW", workers=workers)
        res = O.filtered_solve_blocks(mats, verts, O.rhs_planewave(verts, spec.k, angles), M, 1e-10)
        out.update({f"p{i}_cols": w, f"p{i}_rows": rows, f"p{i}_x": res["x"][rows], f"p{i}_x_full": res["x_full"][rows],
                    f"p{i}_sigma": res["sigma"], f"p{i}_rank": np.int64(res["rank"]),
                    f"p{i}_kappa": np.float64(res["kappa"]), f"p{i}_N": np.int64(spec.N)})
    np.savez(os.path.join(HERE, "c4_batch_subsample.npz"), count=np.int64(C4_COUNT), **out)
    return dict(name="c4_batch_subsample", count=C4_COUNT, seconds={"total": time.perf_counter() - t0},
                N=[int(out[f"p{i}_N"]) for i in range(C4_COUNT)],
                kappa=[float(out[f"p{i}_kappa"]) for i in range(C4_COUNT)])


def run_general(workers):
    """Non-equal-chord mesh: the perturbed circle r = 2 + 0.2 sin 8t (Table I) at N = 2008 vertices
    uniform in the polar angle, k = 0.4, n = 201, tol 1e-3, right-hand sides the line source at
    (3, 0) and four plane waves.  The literal route (dense G^-1/2, eigendecomposition of L~, SVD
    of P C2; Sec. III-A, IV): solutions at 256 seeded rows, the uncompressed filtered solution
    there, v = G^-1 S G^-1 f there, sigma (first n), rank."""
    from oracle import bem_oracle as O
    from paper_2210_08580_gb300 import inputs as I
    t0 = time.perf_counter()
    N, k, n, tol = 2008, 0.4, 201, 1e-3
    verts, _ = I.parameter_mesh(I.perturbed_circle(), N)
    src = np.array([[3.0, 0.0]])
    angles = I.planewave_angles(4)
    mats = O.assemble(verts, k, "SW", workers=workers)
    t1 = time.perf_counter()
    f = np.concatenate([O.rhs_pointsource(verts, k, src), O.rhs_planewave(verts, k, angles)], axis=1)
    res = O.filtered_solve_literal(mats, verts, f, n, tol)
    G = O.gram(verts)
    vx = np.linalg.solve(G, mats["S"] @ np.linalg.solve(G, f))
    rows = np.sort(np.random.default_rng(2008).choice(N, 256, replace=False))
    name = "general_table1_n2008"
    np.savez(os.path.join(HERE, name + ".npz"), rows=rows, angles=angles, source=src, x=res["x"][rows],
             x_full=res["x_full"][rows], vx=vx[rows], sigma=res["sigma"][:n], rank=np.int64(res["rank"]),
             N=np.int64(N), k=np.float64(k), n=np.int64(n), tol=np.float64(tol))
    return dict(name=name, N=N, k=k, n=n, tol=tol, rank=int(res["rank"]), route="filtered_solve_literal",
                seconds={"assemble": t1 - t0, "rest": time.perf_counter() - t1})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--only", default="", choices=["", "c2", "c3", "c4", "c5", "general"])
    args = ap.parse_args()
    summ_path = os.path.join(HERE, "oracle_runs.json")
    summary = {}
    if os.path.exists(summ_path):
        with open(summ_path) as fh:
            summary = json.load(fh)
    runs = summary.get("runs", {})
    todo = [c for c in configs() if not args.only or c["name"].startswith(args.only)]
    for extra in ("c4", "c5", "general"):
        if not args.only or args.only == extra:
            todo.append(extra)
    for cfg in todo:
        if cfg == "c4":
            r = run_c4(args.workers)
        elif cfg == "c5":
            r = run_c5(args.workers)
        elif cfg == "general":
            r = run_general(args.workers)
        else:
            r = run(cfg, args.workers)
        runs[r["name"]] = r
        print(json.dumps(r), flush=True)
        summary = {"host_cores": os.cpu_count(), "workers": args.workers,
                   "command": "python tests/golden/make_goldens.py --workers %d" % args.workers,
                   "oracle": "oracle/bem_oracle.py filtered_solve_blocks (numpy/scipy FP64)", "runs": runs}
        with open(summ_path, "w") as fh:
            json.dump(summary, fh, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
