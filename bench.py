#!/usr/bin/env python
"""Benchmark of the filtered-Calderon fast direct solver (2D TE-EFIE) on GB300.

Workload (one GPU; replicas on N GPUs): random 8-harmonic star r = 1 + sum_m a_m cos(m t + p_m)
(seed = rank), N = 16384 equal-chord P1 segments, k = 2, Laplacian filter n = 201 (M = 100),
compression tolerance 1e-10, 1024 incident plane waves at uniform angles.

A step is one pass of the whole hot path on device-resident inputs:
    bem_assemble (S, N) -> filter_apply -> compress_compact -> factor
    -> bem_rhs_planewave (1024 RHS) -> solve_many
value = RHS solved per second including the factorisation (1024 * ranks / step seconds).
The JSON line also carries the factor time, the solve-only throughput, per-kernel times
(CUDA events on the library's stream), the roofline of the dominant kernel, clocks, an
end-to-end number through the Python API with host buffers, and the CPU oracle baseline.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "factor s + RHS solves/s at N=16384: mixed/batched vs FP64 GPU, rel err ≤1e-8"
# GB300 FP32 pipe: 128 lanes per SM, 152 SMs, 2070 MHz maximum SM clock -> 40.3 T
# FP32 operations per second (an FFMA, FADD or FMUL counts as one operation)
FP32_PEAK_TOPS = 152 * 128 * 2.070e9 / 1e12
# FP32 operations per far-field Gauss point of the S/N assembly, which runs in
# double-float arithmetic (df fma = 15 FP32 ops, df mul = 7, df add = 11) on geometry
# scaled by k: node offsets 2 fma (30), u = (k r)^2 1 mul + 1 fma (22), t = (u - u_mid) /
# u_half 1 add + 1 mul (18), J0/4 and -Y0/4 as degree-7 polynomials (the degrees whose
# coefficients are below 1.1e-8 in 5 FP32 fma, the rest in 9 df fma: 140), the two
# lambda-weighted row sums 4 fma (60)
ASM_OPS_PER_POINT = 270
# DRAM bytes (read + write) per launch from ncu captures of the kernels as they stand
# (absent = not captured since the kernel last changed); the summaries are under profiles/
# (the RHS product's from its N = 4096, 1024-RHS capture: reads x 16 (S's slices and the
# right-hand sides' re-reads grow with N^2), writes x 4 (with N nrhs))
TRAFFIC_BYTES = {"k_assemble": 0.0308e9 + 8.6866e9, "tc_rhs_SY": 0.8303e9 * 16 + 0.0845e9 * 4}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


# GB300 FP64 pipe: 2 DFMA per SM per clock (4 FP64 flops), 152 SMs, 2070 MHz -> 1.26 TFLOP/s
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12

# The method's own arithmetic per launch of the split-bf16 products, counted as the complex
# FP64 products they stand for (a complex multiply-add = 8 real flops, real x complex = 4):
#   tc_rhs_SY      v = S Y          8 N^2 nrhs
#   tc_filter_YN   B = Y2 N         8 n N^2
#   tc_filter_QtS  Y1 = Q^T S       4 n N^2   (Q real)
METHOD_DIMS = {"tc_rhs_SY": ("N", "nrhs", "N", 8.0), "tc_filter_YN": ("n", "N", "N", 8.0),
               "tc_filter_QtS": ("n", "N", "N", 4.0)}


def _dims(args, n_modes):
    return {"N": args.N, "nrhs": args.nrhs, "n": n_modes}


def method_flops(name, args, n_modes):
    if name not in METHOD_DIMS:
        return None
    a, b, c, f = METHOD_DIMS[name]
    d = _dims(args, n_modes)
    return f * d[a] * d[b] * d[c]


def tc_gemm_flops(name, N, nrhs, n_modes, r, S):
    """bf16 tensor flops of one split-slice launch: S(S+1)/2 slice pairs, each the real
    products of the parts (2 M Nc K flops per real product)."""
    dims = {"tc_rhs_SY": (N, nrhs, N), "tc_filter_QtS": (n_modes, N, N),
            "tc_filter_YN": (n_modes, N, N)}
    if name not in dims:
        return None
    M, Nc, K = dims[name]
    # real products of the operands' row blocks: complex x complex = three (Gauss's form,
    # blocks Re, Im, Re + Im), complex x real (the real Fourier basis Q of the filter) = two
    parts = 2.0 if name == "tc_filter_QtS" else 3.0
    return S * (S + 1) / 2 * 2.0 * parts * M * Nc * K


# double-float multiply-add on the FP32 pipe (Dekker product, two-sum, renormalisation): 15
# FP32 operations for 2 FP64-equivalent flops
DF_OPS_PER_FMA = 15


def kernel_roofline(name, cnt, ms, args, n_modes, r, quad_points, basis=None, nsteps=1):
    """Roofline entry of one kernel (average launch of the timed region)."""
    avg_s = ms / cnt / 1000.0
    pk = _peaks()
    if name in ("k_dgemm_df", "k_dgemm_df_tri") and basis:
        # the basis iteration's products: the Gram products X^T (G X) and X^T (L X) form
        # 2 N p^2 flops each and Q = X Cf (one launch per step) 2 N p n; the re-orthonormalisation
        # X R^-1 (k_dgemm_df_tri) N p (p + 1), R^-1 being triangular
        p, N, nc = basis["block"], args.N, basis["ncols"]
        if name == "k_dgemm_df_tri":
            fl = float(N) * p * (p + 1)
        else:                                  # one Q = X Cf launch per step among cnt
            fl = ((cnt - nsteps) * 2.0 * N * p * p + nsteps * 2.0 * N * p * nc) / cnt
        ach = fl / avg_s / 1e12
        peak = FP32_PEAK_TOPS * 2.0 / DF_OPS_PER_FMA
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s (FP64-equivalent, double-float on the FP32 pipe)", "frac": ach / peak,
                "traffic": None, "ms_per_launch": 1000 * avg_s, "flops_per_launch": fl,
                "peak_source": f"derived: FP32 pipe (152 SMs x 128 lanes x 2.07 GHz) / {DF_OPS_PER_FMA} ops per "
                               "double-float multiply-add x 2 flops",
                "vs_fp64_pipe": {"peak": FP64_PEAK_TFLOPS, "frac": ach / FP64_PEAK_TFLOPS}}
    if name == "k_chol" and basis:
        # one CTA: p^3 / 6 double-float multiply-adds against one SM's FP32 pipe
        p = basis["block"]
        fl = p ** 3 / 3.0
        ach = fl / avg_s / 1e12
        peak = 128 * 2.070e9 / 1e12 * 2.0 / DF_OPS_PER_FMA
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s (FP64-equivalent, one SM's FP32 pipe)", "frac": ach / peak, "traffic": None,
                "ms_per_launch": 1000 * avg_s, "flops_per_launch": fl,
                "peak_source": "derived: one SM (one CTA) x 128 FP32 lanes x 2.07 GHz / 15 ops x 2 flops",
                "note": "a sequence of p pivot steps, each a block barrier: latency, not the pipe, bounds it"}
    if name == "k_assemble":
        ach = quad_points * ASM_OPS_PER_POINT / avg_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": FP32_PEAK_TOPS,
                "unit": "TOP/s (FP32 pipe)", "frac": ach / FP32_PEAK_TOPS, "traffic": TRAFFIC_BYTES.get(name),
                "ms_per_launch": 1000 * avg_s, "units_per_launch": quad_points, "ops_per_unit": ASM_OPS_PER_POINT,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz"}
    fl = method_flops(name, args, n_modes)
    if fl is None:
        return {"kernel": name, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None, "ms_per_launch": 1000 * avg_s}
    # digit slices per operand: 6, the right-hand-side product 5 (bem_options.rhs_slices default)
    S = 5 if name == "tc_rhs_SY" else 6
    peak = pk.get("bf16_tflops_sustained", 1700.0)
    src = ("of measured (bf16_tflops_sustained)" if "bf16_tflops_sustained" in pk
           else "of fallback (1.7 PFLOP/s sustained)")
    ach = fl / avg_s / 1e12
    emu = tc_gemm_flops(name, args.N, args.nrhs, n_modes, r, S)
    return {"kernel": name, "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": TRAFFIC_BYTES.get(name), "ms_per_launch": 1000 * avg_s, "peak_source": src,
            "work": "the method's complex FP64 product (%s), FP64-equivalent flops" % name,
            "method_flops_per_launch": fl,
            "vs_fp64_pipe": {"peak": FP64_PEAK_TFLOPS, "frac": ach / FP64_PEAK_TFLOPS,
                             "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2.07 GHz"},
            "emulation": {"slice_pairs": S * (S + 1) // 2, "bf16_flops_per_launch": emu,
                          "achieved": emu / avg_s / 1e12, "frac": emu / avg_s / 1e12 / peak,
                          "note": "tensor-pipe occupancy by the split-bf16 digit products (emulation work)"}}


def roofline(rep, args, n_modes, r, quad_points, top=3, basis=None, nsteps=1):
    """(dominant kernel's roofline, the top kernels' rooflines by time per step); nsteps: the
    steps the timing report covers."""
    order = sorted(rep.items(), key=lambda kv: -kv[1][1])
    rows = [kernel_roofline(nm, c, ms, args, n_modes, r, quad_points, basis, nsteps) for nm, (c, ms) in order[:top]]
    # the filter's two products are one step (a4): report Q^T S beside Y2 N when present
    names = [x["kernel"] for x in rows]
    if "tc_filter_YN" in names and "tc_filter_QtS" in rep and "tc_filter_QtS" not in names:
        c, ms = rep["tc_filter_QtS"]
        rows.append(kernel_roofline("tc_filter_QtS", c, ms, args, n_modes, r, quad_points))
    return rows[0], rows


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--N", type=int, default=16384)
    ap.add_argument("--k", type=float, default=2.0)
    ap.add_argument("--M", type=int, default=100)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--nrhs", type=int, default=1024)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-overlap", action="store_true",
                    help="compress, factor and the right-hand sides one after another (default: "
                         "bem_factor_rhs_planewave, the right-hand sides on a second stream)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare-fp64", action="store_true",
                    help="skip timing the FP64 path beside the mixed path")
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed steps of the FP64 path (median)")
    ap.add_argument("--fp64-warmup", type=int, default=2)
    ap.add_argument("--mesh", default="equal-chord", choices=["equal-chord", "graded"],
                    help="graded: the same star meshed at polar angles t + 0.2 sin t (chords differ by up to "
                         "1.5x), a non-equal-chord mesh with general G and L (computed filter basis)")
    ap.add_argument("--workload", default="single", choices=["single", "batch"],
                    help="single: one N=16384 star (the headline metric); batch: many uneven stars at once")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--streams", type=int, default=0, help="batch streams (0 = tuned per size bucket)")
    ap.add_argument("--batch-solve", default="each", choices=["each", "grouped"],
                    help="batch solves: per problem on its stream, or one persistent launch after all "
                         "right-hand sides")
    return ap.parse_args()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            # nvidia-smi takes a moment to start: let its first sample land before the timed
            # region begins, so that the samples span the region (at most 3 s)
            t0 = time.perf_counter()
            while os.path.getsize(self.path) == 0 and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle
def oracle_measured(N: int, nrhs: int, k: float, M: int, tol: float, seed: int = 0, cols: int = 256,
                    rhs_sample: int = 64, fit_sizes=(1024, 2048), workers: int | None = None) -> dict:
    """The CPU oracle (block route of oracle/bem_oracle.py) timed on the workload, bounded:

    assembly   measured at the full N on the same curve: the oracle's column-block assembly
               of ``cols`` evenly spaced segment columns (each holds N segment pairs) on all
               host cores, scaled by N / cols;
    RHS f      measured at the full N: ``rhs_sample`` of the nrhs plane waves, scaled by
               nrhs / rhs_sample;
    the rest   the block route after the assembly (G^-1 S G^-1 f for all nrhs, filter block,
               compression, Woodbury solve of all nrhs) timed end to end at two smaller N of
               the same curve family and extrapolated as c N^p with p fitted from the two.
    Returns the per-phase seconds (measured and estimated) and the estimate of one full step."""
    import multiprocessing as mp

    from oracle import bem_oracle as O
    from paper_2210_08580_gb300 import inputs as I
    workers = workers or cpu_cores()
    curve = I.random_star(seed)
    verts, _, _ = I.equal_chord_mesh(curve, N)
    out = {"N": N, "nrhs": nrhs, "workers": workers}
    block = 8
    starts = np.linspace(0, N - block, cols // block).astype(int)
    with mp.get_context("spawn").Pool(workers) as pool:
        list(O.assembled_column_blocks(verts, k, [0], 1, "SW", pool=pool))        # start the workers
        t0 = time.perf_counter()
        for _ in O.assembled_column_blocks(verts, k, starts, block, "SW", pool=pool):
            pass
        t_asm = time.perf_counter() - t0
        out["assemble_sample_s"] = t_asm
        out["assemble_cols"] = len(starts) * block
        out["assemble_s"] = t_asm * N / (len(starts) * block)
        t0 = time.perf_counter()
        O.rhs_planewave(verts, k, I.planewave_angles(nrhs)[:rhs_sample])
        out["rhs_sample_s"] = time.perf_counter() - t0
        out["rhs_s"] = out["rhs_sample_s"] * nrhs / rhs_sample
        rest = []
        for Ns in fit_sizes:
            v_s, _, _ = I.equal_chord_mesh(curve, Ns)
            mats = O.assemble(v_s, k, "SW", pool=pool)
            f = O.rhs_planewave(v_s, k, I.planewave_angles(nrhs))
            t0 = time.perf_counter()
            O.filtered_solve_blocks(mats, v_s, f, min(M, (Ns - 2) // 4), tol)
            rest.append(time.perf_counter() - t0)
    p = math.log(rest[1] / rest[0]) / math.log(fit_sizes[1] / fit_sizes[0])
    out["rest_fit"] = {"sizes": list(fit_sizes), "seconds": rest, "exponent": p}
    out["rest_s"] = rest[1] * (N / fit_sizes[1]) ** p
    out["step_s"] = out["assemble_s"] + out["rhs_s"] + out["rest_s"]
    return out


def oracle_sample_text(m: dict, golden=None) -> str:
    txt = (f"oracle block route (numpy/scipy FP64, {m['workers']} processes) on the same workload: assembly "
           f"measured at N={m['N']} on {m['assemble_cols']} of "
           f"{m['N']} segment columns ({m['assemble_sample_s']:.1f} s, scaled to {m['assemble_s']:.0f} s); "
           f"plane-wave RHS measured at N={m['N']} for a sample ({m['rhs_sample_s']:.2f} s, scaled to "
           f"{m['rhs_s']:.1f} s for {m['nrhs']}); filter block + compression + {m['nrhs']}-RHS solve timed at "
           f"N={m['rest_fit']['sizes']} ({', '.join('%.2f' % x for x in m['rest_fit']['seconds'])} s), fitted "
           f"N^{m['rest_fit']['exponent']:.2f} -> {m['rest_s']:.1f} s; step {m['step_s']:.0f} s")
    if golden:
        txt += (f"; the full C3 oracle run of tests/golden/make_goldens.py took {golden['total_s']:.0f} s "
                f"(assembly {golden['assemble_s']:.0f} s) on {golden['workers']} processes of a "
                f"{golden['host_cores']}-core host")
    return txt


def golden_c3_run():
    """Wall time of the committed full-size C3 oracle run (tests/golden/oracle_runs.json)."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "oracle_runs.json")) as fh:
            d = json.load(fh)
        r = d["runs"]["c3_random_star0_n16384"]["seconds"]
        return {"assemble_s": r["assemble"], "total_s": sum(r.values()), "workers": d["workers"],
                "host_cores": d["host_cores"]}
    except Exception:
        return None


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ----------------------------------------------------------------------------- replicas
def replica_seed(rank: int) -> int:
    """Each rank solves its own star (independent problems, no data-path collective)."""
    return rank


def reduce_max(x: float, dist=None, device=None) -> float:
    """Maximum of a per-rank time over all ranks (identity on one rank)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds


# ----------------------------------------------------------------------------- main
def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands, timed on the host cores.  Each step is one
    bounded measurement of the oracle on the workload (oracle_measured); value = nrhs over
    the oracle's time for one full step."""
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_measured(args.N, args.nrhs, args.k, args.M, args.tol, cols=64, rhs_sample=16, fit_sizes=(384, 768))
    rates, times, last = [], [], None
    for _ in range(args.steps):
        t = time.perf_counter()
        last = oracle_measured(args.N, args.nrhs, args.k, args.M, args.tol)
        times.append(time.perf_counter() - t)
        rates.append(args.nrhs / last["step_s"])
    val = statistics.median(rates)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "RHS/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.median(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"value": val, "unit": "RHS/s", "cores": last["workers"], "kind": "oracle",
                             "sample": oracle_sample_text(last, golden_c3_run())},
            "e2e": {"value": val, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch(args, rank, world):
    """Many uneven problems at once (random stars, N ~ U{512..8192}, k = 10^U(-2, log10 5),
    64..512 plane waves each): every problem assembled, filtered, compressed, factored,
    its right-hand sides formed and solved; value = right-hand sides solved per second."""
    import torch
    dist = None
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2210_08580_gb300 import batch, inputs as I
    specs = I.batch_problems(count=args.batch_count, first_seed=100 + 1000 * rank)
    problems = batch.problems_from_inputs(specs)
    nrhs_total = sum(len(p.angles) for p in problems)
    tiles = batch.autotune_tiles(problems, device=local, reps=1) if args.prec == "mixed" else None
    if args.streams > 0:
        n_streams = args.streams
        tuned = None
    else:
        tuned = batch.autotune_streams(problems, prec=args.prec, device=local, candidates=(1, 2, 4, 8), sample=4)
        n_streams = max(set(tuned.values()), key=list(tuned.values()).count)
    solve = args.batch_solve
    bs = batch.BatchSolver(problems, prec=args.prec, device=local, n_streams=n_streams, tiles=tiles, solve=solve)
    for _ in range(args.warmup):
        bs.run()
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        res = bs.run()
    torch.cuda.synchronize(dev)
    dt = reduce_max((time.perf_counter() - t0) / args.steps, dist, dev)
    clk = clocks.stop()
    solve_stage = time_solve_stage(bs, res, dev)
    bs.close()
    if rank == 0:
        line = {"metric": "batched factor + RHS solves/s, uneven random stars", "value": job_value(nrhs_total, world, dt),
                "unit": "RHS/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1000 * dt, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.prec == "fp64" else "bf16-split+f64", "data": "synthetic",
                "config": {"workload": f"{args.batch_count} random stars (seeds 100.., N ~ U{{512..8192}}, "
                                       f"k = 10^U(-2, log10 5), 64..512 plane waves)",
                           "problems": args.batch_count, "rhs_total": nrhs_total, "prec": args.prec,
                           "streams": n_streams, "tuned_streams": tuned, "solve": solve,
                           "tuned_tiles": {str(b): {k: v for k, v in c.items() if k != "times_ms"}
                                           for b, c in (tiles or {}).items()},
                           "assembly": "one persistent launch over a global tile queue (bem_assemble_batch)",
                           "solve_stage": solve_stage,
                           "parallelism": f"replicas x{world}"},
                "clocks": clk}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def time_solve_stage(bs, res, dev, reps=3):
    """The FP64 Woodbury solves of every problem of a factored batch, two ways: the CUDA
    graph of one solve_many_noalloc per problem (SolveGraph) and one persistent launch over
    all problems' tiles (solve_grouped).  Wall time per solve of the whole batch, synchronised
    on both sides (after one untimed run of each); the two results' largest relative
    difference; FP64 flops of the method's products (8 per complex multiply-add:
    V^H v, Kinv T, U T2)."""
    import torch
    from paper_2210_08580_gb300 import batch
    vs = [out["v"] for out in res]
    flops = sum(8.0 * out["v"].shape[0] * (2.0 * out["rank"] * out["v"].shape[1] + out["rank"] ** 2)
                for out in res)
    xs = [torch.empty_like(v) for v in vs]
    runs = [("grouped", lambda: batch.solve_grouped(bs.solvers, vs, xs))]
    try:
        g = batch.SolveGraph(bs, device=dev.index)
        for i, v in enumerate(vs):
            g.v[i].copy_(v)
        runs.insert(0, ("graph", g.replay))
    except Exception as e:          # e.g. rank x nrhs above solve_many_noalloc's fixed scratch
        g = None
        graph_error = str(e)
    timed = {"graph": None}
    s0 = bs.solvers[0]
    kernel_ms = None
    for name, fn in runs:
        fn()
        torch.cuda.synchronize(dev)
        if name == "grouped":
            s0.timing(True)
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize(dev)
        timed[name] = (time.perf_counter() - t0) / reps
        if name == "grouped":
            cnt, tot = s0.timing_report().get("k_woodbury_batch", [0, 0.0])
            s0.timing(False)
            kernel_ms = tot / cnt if cnt else None
    roof = None
    if kernel_ms:
        ach = flops / (kernel_ms / 1000.0) / 1e12
        roof = {"kernel": "k_woodbury_batch", "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s (FP64 pipe)", "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                "ms_per_launch": kernel_ms, "flops_per_launch": flops,
                "peak_source": "derived: 152 SMs x 2 DFMA per clock x 2 flops x 2.07 GHz"}
    if g is None:
        return {"graph_ms": None, "graph_error": graph_error, "grouped_ms": round(1000 * timed["grouped"], 3),
                "fp64_gflop": round(flops / 1e9, 2)}
    diff = max(float((a - b).abs().max() / b.abs().max()) for a, b in zip(xs, g.x))
    return {"graph_ms": round(1000 * timed["graph"], 3), "grouped_ms": round(1000 * timed["grouped"], 3),
            "fp64_gflop": round(flops / 1e9, 2),
            "grouped_fp64_tflops": round(flops / timed["grouped"] / 1e12, 3),
            "max_rel_diff": diff, "reps": reps, "roofline": roof,
            "how": "one solve of every problem's right-hand sides: CUDA graph of per-problem "
                   "solve_many_noalloc vs one persistent launch (bem_solve_batch)"}


def workload_config(args):
    mesh = ("" if args.mesh == "equal-chord" else
            ", mesh at polar angles t + 0.2 sin t (non-equal chords: general G, L, computed filter basis)")
    return {"workload": f"random 8-harmonic star (seed=rank), N={args.N}, k={args.k}, n={2 * args.M + 1}, "
                        f"tol={args.tol}, {args.nrhs} plane waves{mesh}", "mesh": args.mesh,
            "N": args.N, "k": args.k, "n_modes": 2 * args.M + 1, "tol": args.tol, "nrhs": args.nrhs,
            "prec": args.prec, "parallelism": f"replicas x{args.gpus}",
            "schedule": ("compress, factor, right-hand sides in turn" if args.no_overlap else
                         "right-hand sides on a second stream beside compress and factor"),
            "l2": "working set > L2: S and N (4.3 GB each at N=16384) are rewritten and read every step"}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batch":
        return run_batch(args, rank, world)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2210_08580_gb300 import bem, inputs as I

    if args.mesh == "graded":
        verts_np, _ = I.parameter_mesh(I.random_star(replica_seed(rank)), args.N, grade=0.2)
    else:
        verts_np, _, _ = I.equal_chord_mesh(I.random_star(replica_seed(rank)), args.N)
    ang_np = I.planewave_angles(args.nrhs)
    verts = torch.from_numpy(verts_np).to(dev)
    ang = torch.from_numpy(ang_np).to(dev)
    n_modes = 2 * args.M + 1
    stream = torch.cuda.current_stream(dev)
    s = bem.Solver(device=local, prec=args.prec, stream=stream)
    v = torch.empty((args.nrhs, args.N), dtype=torch.complex128, device=dev)
    x = torch.empty_like(v)
    info = {}

    def factor_and_rhs(sv, ang_in, v_out):
        """compression, factor and right-hand sides: overlapped in one call, or one after another"""
        if args.no_overlap:
            r = sv.compress(args.tol)
            sv.factor()
            sv.L.bem_rhs_planewave(sv.h, ang_in.data_ptr(), args.nrhs, None, v_out.data_ptr(), args.N)
            return r
        r = ctypes.c_int64()
        sv._check(sv.L.bem_factor_rhs_planewave(sv.h, float(args.tol), ang_in.data_ptr(), args.nrhs, None,
                                                v_out.data_ptr(), args.N, ctypes.byref(r)))
        return r.value

    def step(verts_in, ang_in, x_out=None):
        s.assemble(verts_in, args.k, ops="SW")
        s.filter_apply(n_modes)
        info["r"] = factor_and_rhs(s, ang_in, v)
        s.solve(v, out=x if x_out is None else x_out)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step(verts, ang)
    barrier()

    # ---- timed region (device-resident inputs)
    clocks = ClockSampler(local)
    clocks.start()
    s.timing(True)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(verts, ang)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    rep = s.timing_report()
    s.timing(False)
    clk = clocks.stop()
    ms = reduce_max(ms, dist, dev)
    ms_step = ms / args.steps
    value = job_value(args.nrhs, world, ms_step / 1000.0)

    # ---- phase split of one extra instrumented step (factor vs RHS vs solve, one after another)
    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream); fn(); b.record(stream); torch.cuda.synchronize(dev)
        return a.elapsed_time(b)
    s.timing(True)              # the kernels of this step run alone (no overlap)
    t_fac = timed(lambda: (s.assemble(verts, args.k, ops="SW"), s.filter_apply(n_modes),
                           s.compress(args.tol), s.factor()))
    t_rhs = timed(lambda: s.L.bem_rhs_planewave(s.h, ang.data_ptr(), args.nrhs, None, v.data_ptr(), args.N))
    t_sol = timed(lambda: s.solve(v, out=x))
    rep_alone = s.timing_report()
    s.timing(False)
    _, iters, resid = s.solve(v, report=True, out=x)

    # ---- roofline of the dominant kernel
    launches = sum(c for c, _ in rep.values())
    sinfo = s.info()
    quad_points = sinfo["quad_points"]
    basis = None
    if not sinfo["equal_chord"]:
        basis = {"block": sinfo["basis_block"], "iters": sinfo["basis_iters"],
                 "ncols": n_modes}                   # the bench keeps the kernel mode (default)
    roof, roofs = roofline(rep, args, n_modes, info["r"], quad_points, basis=basis, nsteps=args.steps)
    # the same rooflines with every kernel running alone (the phase-split step): in the timed
    # steps the right-hand-side product shares its SMs with the compression and factor
    _, roofs_alone = roofline(rep_alone, args, n_modes, info["r"], quad_points, basis=basis, nsteps=1)

    # ---- end to end through the Python API with host buffers.  Every step copies its inputs
    # from pinned host memory and its solution back to pinned host memory inside the timed
    # region; the solution's copy runs on a copy stream while the next step assembles (two
    # solution buffers on each side, ordered by events), as a solve service would pipeline it.
    e2e = None
    if not args.no_e2e:
        vh = torch.from_numpy(verts_np).pin_memory()
        ah = torch.from_numpy(ang_np).pin_memory()
        xhs = [torch.empty((args.nrhs, args.N), dtype=torch.complex128).pin_memory() for _ in range(2)]
        xds = [x, torch.empty_like(x)]
        copy_stream = torch.cuda.Stream(dev)
        copied = [None, None]

        def e2e_step(it):
            b = it % 2
            vd = vh.to(dev, non_blocking=True)
            ad = ah.to(dev, non_blocking=True)
            if copied[b] is not None:
                stream.wait_event(copied[b])        # the copy that read xds[b] has finished
            step(vd, ad, xds[b])
            solved = torch.cuda.Event()
            solved.record(stream)
            copy_stream.wait_event(solved)
            with torch.cuda.stream(copy_stream):
                xhs[b].copy_(xds[b], non_blocking=True)
            copied[b] = torch.cuda.Event()
            copied[b].record(copy_stream)

        for it in range(2):                         # one untimed pass through both buffers
            e2e_step(it)
        barrier()
        t0 = time.perf_counter()
        marks = []
        for it in range(args.steps):
            e2e_step(it)
            marks.append(time.perf_counter())       # host time when the step's work is enqueued
        barrier()
        t1 = time.perf_counter()
        e2e_s = reduce_max((t1 - t0) / args.steps, dist, dev)
        # per-step host intervals (the compression's rank read-back makes each step wait for
        # the device, so these follow the device's progress up to one step of lag)
        per = [1000.0 * (b - a) for a, b in zip([t0] + marks[:-1], marks)]
        e2e = {"value": job_value(args.nrhs, world, e2e_s), "unit": "RHS/s",
               "h2d_bytes_per_step": int(vh.numel() * 8 + ah.numel() * 8),
               "d2h_bytes_per_step": int(xhs[0].numel() * 16),
               "ms_per_step": 1000.0 * e2e_s, "host_ms_per_step_all": [round(v, 3) for v in per],
               "drain_ms": round(1000.0 * (t1 - marks[-1]), 3) if marks else None}

    fp64_cmp = None
    if not args.no_compare_fp64 and args.prec == "mixed":
        # the same step on the FP64 path (warm-up, then the median of timed steps, with its
        # per-kernel split), and the metric's accuracy bar: the mixed solution against the
        # FP64 one on identical inputs (max over RHS of the relative error)
        x_mixed = x.clone()
        v64 = torch.empty_like(v)
        x64 = torch.empty_like(x)
        s64 = bem.Solver(device=local, prec="fp64", stream=stream)

        def step64():
            s64.assemble(verts, args.k, ops="SW")
            s64.filter_apply(n_modes)
            r64 = factor_and_rhs(s64, ang, v64)
            s64.solve(v64, out=x64)
            return r64

        for _ in range(args.fp64_warmup):
            step64()
        torch.cuda.synchronize(dev)
        s64.timing(True)
        t64s = [timed(step64) for _ in range(args.fp64_steps)]
        rep64 = s64.timing_report()
        s64.timing(False)
        t64 = statistics.median(t64s)
        err = ((x_mixed - x64).abs().amax(dim=1) / x64.abs().amax(dim=1)).max().item()
        k64 = {k_: round(v_[1] / args.fp64_steps, 3) for k_, v_ in rep64.items()}
        zg = rep64.get("gemm_rhs_SY")
        zgemm_roof = None
        if zg:
            fl = 8.0 * args.N * args.N * args.nrhs
            ach = fl / (zg[1] / zg[0] / 1000.0) / 1e12
            zgemm_roof = {"kernel": "k_zgemm (gemm_rhs_SY)", "bound": "fp64", "achieved": ach,
                          "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                          "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2.07 GHz"}
        fp64_cmp = {"ms_per_step": t64, "steps": args.fp64_steps, "warmup": args.fp64_warmup,
                    "ms_per_step_all": t64s, "value": args.nrhs / (t64 / 1000.0), "unit": "RHS/s",
                    "kernels_ms_per_step": k64, "rhs_product_roofline": zgemm_roof,
                    "mixed_rel_err_vs_fp64": err, "bar": 1e-8, "pass": bool(err <= 1e-8)}
        s64.close()
        del v64, x64, x_mixed

    cpu = None
    # the oracle's measured leg is its block route, which takes equal-chord meshes only
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.mesh == "equal-chord":
        m = oracle_measured(args.N, args.nrhs, args.k, args.M, args.tol)
        cpu = {"value": args.nrhs / m["step_s"], "unit": "RHS/s", "cores": m["workers"], "kind": "oracle",
               "sample": oracle_sample_text(m, golden_c3_run()), "phases_s": {
                   "assemble": m["assemble_s"], "rhs": m["rhs_s"], "rest": m["rest_s"]},
               "rest_fit": m["rest_fit"]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if args.prec == "fp64" else "bf16-split+f64",
                "data": "synthetic", "config": workload_config(args),
                "factor_s": t_fac / 1000.0, "rhs_s": t_rhs / 1000.0, "solve_s": t_sol / 1000.0,
                "solve_rhs_per_s": args.nrhs / (t_sol / 1000.0), "rank": info["r"],
                "max_rel_residual": resid, "refine_iters": iters,
                "kernels_ms_per_step": {k_: round(v_[1] / args.steps, 3) for k_, v_ in rep.items()},
                "roofline": roof, "rooflines": roofs, "rooflines_alone": roofs_alone, "clocks": clk, "gpu_launches": launches, "e2e": e2e, "cpu_baseline": cpu}
        if fp64_cmp:
            line["fp64_path"] = fp64_cmp
        if basis:
            line["config"]["filter_basis"] = {"block": basis["block"], "shift_invert_steps": basis["iters"]}
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
