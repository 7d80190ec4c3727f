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

and a summary with the oracle's wall time per phase and the host's core count in
``tests/golden/oracle_runs.json``.

Configurations: star r = 1 + 0.3 cos 5t, N = 4096, k in {1e-3, 1e-2, 1e-1, 1, 5}, n = 201,
tol 1e-10 (256 plane waves); random 8-harmonic star of seed 0, N = 16384, k = 2, n = 201,
tol 1e-10 (1024 plane waves).

    python tests/golden/make_goldens.py [--workers W] [--only c2|c3]
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
    np.savez(os.path.join(HERE, cfg["name"] + ".npz"), rows=rows, angles=angles, x=res["x"][rows],
             x_full=res["x_full"][rows], vx=res["vx"][rows], xnorm_G=G_norm, sigma=res["sigma"],
             rank=np.int64(res["rank"]), kappa=np.float64(res["kappa"]), N=np.int64(N), k=np.float64(cfg["k"]),
             M=np.int64(cfg["M"]), tol=np.float64(cfg["tol"]))
    xr = res["x"]
    comp_err = float(np.max(np.abs(xr - res["x_full"])) / np.max(np.abs(res["x_full"])))
    return dict(name=cfg["name"], N=N, k=cfg["k"], n=2 * cfg["M"] + 1, tol=cfg["tol"], rank=res["rank"],
                kappa=res["kappa"], compressed_vs_uncompressed=comp_err, seconds=t)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--only", default="", choices=["", "c2", "c3"])
    args = ap.parse_args()
    summ_path = os.path.join(HERE, "oracle_runs.json")
    summary = {}
    if os.path.exists(summ_path):
        with open(summ_path) as fh:
            summary = json.load(fh)
    runs = summary.get("runs", {})
    for cfg in configs():
        if args.only and not cfg["name"].startswith(args.only):
            continue
        r = run(cfg, args.workers)
        runs[cfg["name"]] = r
        print(json.dumps(r), flush=True)
        summary = {"host_cores": os.cpu_count(), "workers": args.workers,
                   "command": "python tests/golden/make_goldens.py --workers %d" % args.workers,
                   "oracle": "oracle/bem_oracle.py filtered_solve_blocks (numpy/scipy FP64)", "runs": runs}
        with open(summ_path, "w") as fh:
            json.dump(summary, fh, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
