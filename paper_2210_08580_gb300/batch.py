"""Many geometries at once: the batching layer.

A batch of independent problems (uneven N, k and numbers of incident waves) is spread
over several CUDA streams, one host thread per stream (the C calls release the GIL), so
that the kernels of small problems fill the GPU side by side.  The cooperative kernels of
the compression and the Woodbury core (grid barriers that need every CTA resident) draw
on a budget of one CTA per SM: a problem enters that phase only when the CTAs of its
largest cooperative grid fit in what the running ones leave, so every grid of the phase
is resident at once (a problem whose grid alone exceeds the budget waits for an idle GPU
and runs alone); its stream is synchronised before the budget is returned.  Everything
else overlaps freely.

``autotune_streams`` times a few stream counts on a sample of the batch and keeps the
fastest per problem-size bucket.  ``SolveGraph`` records the FP64 Woodbury solves of every
problem (``solve_many_noalloc``, which allocates nothing) into one CUDA graph, replayed
for each new set of right-hand sides; ``solve_grouped`` instead solves every problem's
right-hand sides in ONE persistent launch (``bem_solve_batch``: tiles of all problems'
Woodbury products from a global queue, bounded device-side waits between the stages).

By default the assembly stage of all problems is one persistent launch
(``bem_assemble_batch``): CTAs take tiles from a global queue over every problem, largest
first, so the tiles of small problems fill the GPU beside those of large ones.  Each problem
is solved by exactly the kernels a single ``bem.Solver`` uses (the batched assembly runs the
same tile code), so the results are those of the problems solved one after another.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import threading
import time

import numpy as np
import torch

from . import bem, inputs


@dataclasses.dataclass
class Problem:
    verts: np.ndarray          # (N, 2) closed counter-clockwise polygon, equal chords
    k: float
    angles: np.ndarray         # plane-wave incidence angles (nrhs,)
    n_modes: int               # filter modes n = 2M + 1
    tol: float = 1e-10


def problems_from_inputs(specs, tol: float = 1e-10) -> list[Problem]:
    """Problems of ``inputs.batch_problems``: n = min(201, 2 floor(N/8) + 1)."""
    out = []
    for s in specs:
        v, _, _ = inputs.equal_chord_mesh(s.curve, s.N)
        out.append(Problem(verts=v, k=s.k, angles=inputs.planewave_angles(s.nrhs),
                           n_modes=min(201, 2 * (s.N // 8) + 1), tol=tol))
    return out


def size_bucket(N: int) -> int:
    """Problem-size bucket for the tuner: log2 of N rounded down."""
    return int(math.log2(max(N, 1)))


class BatchSolver:
    """Solves a list of Problems concurrently on ``n_streams`` streams of one device."""

    def __init__(self, problems: list[Problem], prec: str = "mixed", device: int = 0, n_streams: int = 4,
                 refine_rtol: float = 1e-10, persistent: bool = True, tiles: dict | None = None,
                 solve: str = "each"):
        """persistent: assemble every problem's S and N in one launch over a global tile queue
        (bem_assemble_batch) before the per-problem stages; False: each problem assembles on
        its own stream.  tiles: {size bucket: tile options} from ``autotune_tiles`` (mixed
        path), applied to each problem by its bucket.  solve: "each" solves every problem on
        its stream as soon as its right-hand sides are formed (the results of one-by-one
        solves, bit for bit); "grouped" solves all problems after the last right-hand sides
        in one persistent launch of FP64 Woodbury tiles (``solve_grouped``: the one-by-one
        FP64 solves up to the order of the sums; on mixed handles the exact inverse of the
        compressed operator, without refinement)."""
        if solve not in ("each", "grouped"):
            raise ValueError("solve: 'each' or 'grouped'")
        self.solve = solve
        self.problems = problems
        self.prec = prec
        self.device = device
        self.n_streams = max(1, int(n_streams))
        self.refine_rtol = refine_rtol
        self.persistent = persistent
        self.tiles = tiles or {}
        self.streams = [torch.cuda.Stream(device=device) for _ in range(self.n_streams)]
        self._coop = threading.Condition()
        props = torch.cuda.get_device_properties(device)
        self.nsm = props.multi_processor_count
        self._budget = self.nsm
        self.solvers: list[bem.Solver | None] = [None] * len(problems)
        self.results: list[dict | None] = [None] * len(problems)

    def _solver(self, i: int, stream: torch.cuda.Stream) -> bem.Solver:
        s = self.solvers[i]
        if s is None:
            tiles = self.tiles.get(size_bucket(self.problems[i].verts.shape[0])) if self.prec == "mixed" else None
            s = bem.Solver(device=self.device, prec=self.prec, stream=stream, refine_rtol=self.refine_rtol,
                           tiles=tiles)
            self.solvers[i] = s
        return s

    def _one(self, i: int, stream: torch.cuda.Stream, assembled: bool = False):
        p = self.problems[i]
        dev = torch.device("cuda", self.device)
        with torch.cuda.stream(stream):
            s = self._solver(i, stream)
            ang = torch.from_numpy(np.ascontiguousarray(p.angles)).to(dev, non_blocking=True)
            if not assembled:
                verts = torch.from_numpy(np.ascontiguousarray(p.verts)).to(dev, non_blocking=True)
                s.assemble(verts, p.k, ops="SW")
            s.filter_apply(p.n_modes)
            need = self._coop_ctas(p)
            with self._coop:
                self._coop.wait_for(lambda: self._budget >= need)
                self._budget -= need
            try:
                r = s.compress(p.tol)          # synchronises the stream (returns the rank)
                s.factor()
                stream.synchronize()
            finally:
                with self._coop:
                    self._budget += need
                    self._coop.notify_all()
            v = s.rhs_planewave(ang)
            x = s.solve(v) if self.solve == "each" else None
            self.results[i] = dict(x=x, v=v, rank=r)

    def _coop_ctas(self, p: Problem) -> int:
        """CTAs of the problem's largest cooperative grid (QR, Jacobi, Gauss-Jordan), capped
        at the budget (such a problem then runs its phase alone)."""
        N, n = p.verts.shape[0], p.n_modes
        qr = min(self.nsm, (N + 15) // 16)
        jac = (n + 1) // 2
        gj = max(1, (2 * n + 2) // 3)
        return min(self.nsm, max(qr, jac, gj))

    def run(self) -> list[dict]:
        """Assemble, filter, compress, factor, form the RHS and solve every problem; returns
        per problem dict(x=(nrhs, N) complex128, v=..., rank=r)."""
        order = sorted(range(len(self.problems)), key=lambda i: -self.problems[i].verts.shape[0])
        queues = [order[q::self.n_streams] for q in range(self.n_streams)]
        errors = []
        if self.persistent:
            dev = torch.device("cuda", self.device)
            sv = []
            for q in range(self.n_streams):
                for i in queues[q]:
                    sv.append((i, self._solver(i, self.streams[q])))
            bem.assemble_batch([s for _, s in sv],
                               [torch.from_numpy(np.ascontiguousarray(self.problems[i].verts)).to(dev) for i, _ in sv],
                               [self.problems[i].k for i, _ in sv])

        def worker(q):
            try:
                for i in queues[q]:
                    self._one(i, self.streams[q], assembled=self.persistent)
                self.streams[q].synchronize()
            except Exception as e:          # re-raised on the calling thread
                errors.append(e)

        threads = [threading.Thread(target=worker, args=(q,)) for q in range(self.n_streams)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        if errors:
            raise errors[0]
        if self.solve == "grouped":
            xs = solve_grouped(self.solvers, [r["v"] for r in self.results])
            for r, x in zip(self.results, xs):
                r["x"] = x
        return self.results

    def close(self):
        for s in self.solvers:
            if s is not None:
                s.close()
        self.solvers = [None] * len(self.problems)


def autotune_streams(problems: list[Problem], prec: str = "mixed", device: int = 0,
                     candidates=(1, 2, 4, 8), sample: int = 8) -> dict:
    """Times ``BatchSolver.run`` on up to ``sample`` problems of each size bucket for every
    stream count in ``candidates``; returns {bucket: best stream count}."""
    buckets: dict[int, list[Problem]] = {}
    for p in problems:
        buckets.setdefault(size_bucket(p.verts.shape[0]), []).append(p)
    best = {}
    for b, ps in sorted(buckets.items()):
        ps = ps[:sample]
        times = {}
        for c in candidates:
            bs = BatchSolver(ps, prec=prec, device=device, n_streams=min(c, len(ps)))
            bs.run()                           # warm-up (allocations, tables)
            torch.cuda.synchronize(device)
            t0 = time.perf_counter()
            bs.run()
            torch.cuda.synchronize(device)
            times[c] = time.perf_counter() - t0
            bs.close()
        best[b] = min(times, key=times.get)
    return best


# candidate tile shapes (tile width, K splits; 0 = the library's own choice) per stage of the
# mixed path's split-bf16 products
TILE_CANDIDATES = {
    "filter": ((0, 0), (112, 0), (128, 0), (112, 1), (128, 1), (112, 2), (112, 4)),
    "rhs": ((0, 0), (128, 1), (128, 2), (128, 4), (112, 1), (112, 2)),
}
_STAGE_KERNELS = {"filter": ("tc_filter_QtS", "tc_filter_YN", "k_splitk_reduce"),
                  "rhs": ("tc_rhs_SY", "k_splitk_reduce")}


def _stage_ms(p: Problem, stage: str, bn: int, sk: int, device: int, reps: int) -> float:
    """Kernel time of one stage of the mixed path on problem p with the given tile shape."""
    dev = torch.device("cuda", device)
    s = bem.Solver(device=device, prec="mixed", tiles={f"{stage}_tile_n": bn, f"{stage}_split_k": sk})
    try:
        s.assemble(torch.from_numpy(np.ascontiguousarray(p.verts)).to(dev), p.k, ops="SW")
        ang = torch.from_numpy(np.ascontiguousarray(p.angles)).to(dev)
        best = float("inf")
        for _ in range(reps + 1):                # the first pass warms up (allocations)
            s.timing(True)
            if stage == "filter":
                s.filter_apply(p.n_modes)
            else:
                s.rhs_planewave(ang)
            rep = s.timing_report()
            s.timing(False)
            best = min(best, sum(rep.get(k, (0, 0.0))[1] for k in _STAGE_KERNELS[stage]))
        return best
    finally:
        s.close()


def autotune_tiles(problems: list[Problem], device: int = 0, candidates: dict | None = None,
                   reps: int = 2) -> dict:
    """The batching layer's tile-shape tuner: for each size bucket it takes the bucket's largest
    problem, times every candidate (tile width, K splits) of each stage's split-bf16 products
    (the filter products Q^T S, Y2 N; the right-hand-side product S Y) by the kernels' own
    events, and keeps the fastest.  Returns {bucket: {"filter_tile_n", "filter_split_k",
    "rhs_tile_n", "rhs_split_k"}, with "times_ms": {stage: {candidate: ms}}}."""
    cands = candidates or TILE_CANDIDATES
    buckets: dict[int, Problem] = {}
    for p in problems:
        b = size_bucket(p.verts.shape[0])
        if b not in buckets or p.verts.shape[0] > buckets[b].verts.shape[0]:
            buckets[b] = p
    out = {}
    for b, p in sorted(buckets.items()):
        choice, times = {}, {}
        for stage, cs in cands.items():
            t = {c: _stage_ms(p, stage, c[0], c[1], device, reps) for c in cs}
            bn, sk = min(t, key=t.get)
            choice[f"{stage}_tile_n"] = bn
            choice[f"{stage}_split_k"] = sk
            times[stage] = {f"{c[0]}x{c[1]}": round(v, 4) for c, v in t.items()}
        choice["times_ms"] = times
        out[b] = choice
    return out


class SolveGraph:
    """One CUDA graph holding the FP64 Woodbury solves x_i = A_i^-1 v_i of every factored
    problem of a BatchSolver (``solve_many_noalloc``: no allocation, so it can be recorded).
    ``replay()`` re-runs all of them on whatever the captured v_i buffers hold now.  The
    solves are recorded one after another on one stream (they share the library's fixed
    scratch array)."""

    def __init__(self, batch: BatchSolver, device: int = 0):
        self.batch = batch
        self.v = []
        self.x = []
        dev = torch.device("cuda", device)
        L = bem.load_library()
        for i, s in enumerate(batch.solvers):
            if s is None:
                raise ValueError("run the batch first")
            nrhs = len(batch.problems[i].angles)
            self.v.append(torch.zeros((nrhs, s.N), dtype=torch.complex128, device=dev))
            self.x.append(torch.zeros((nrhs, s.N), dtype=torch.complex128, device=dev))
        self.stream = torch.cuda.Stream(device=device)
        # first call outside capture (looks up the scratch array), then record
        for i, s in enumerate(batch.solvers):
            L.bem_set_stream(s.h, torch.cuda.current_stream(dev).cuda_stream)
            st = L.solve_many_noalloc(s.h, self.v[i].data_ptr(), s.N, self.x[i].data_ptr(), s.N, self.v[i].shape[0])
            if st != 0:
                raise bem.BemError(st, L.bem_last_error(s.h).decode())
        torch.cuda.synchronize(device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            for i, s in enumerate(batch.solvers):
                L.bem_set_stream(s.h, self.stream.cuda_stream)
                st = L.solve_many_noalloc(s.h, self.v[i].data_ptr(), s.N, self.x[i].data_ptr(), s.N,
                                          self.v[i].shape[0])
                if st != 0:
                    raise bem.BemError(st, L.bem_last_error(s.h).decode())
        for s in batch.solvers:
            L.bem_set_stream(s.h, s.stream.cuda_stream)

    def replay(self):
        self.graph.replay()


def _grouped_args(solvers: list, vs: list, xs: list | None):
    if len(solvers) != len(vs) or not solvers:
        raise ValueError("one right-hand-side block per solver")
    if xs is None:
        xs = [torch.empty_like(v) for v in vs]
    for s, v, x in zip(solvers, vs, xs):
        if v.dtype != torch.complex128 or v.shape != x.shape or v.shape[1] != s.N or not v.is_contiguous() \
                or not x.is_contiguous():
            raise ValueError("v, x: contiguous complex128 (nrhs, N) tensors")
    n = len(solvers)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    ld = (i64 * n)(*[s.N for s in solvers])
    args = ((vp * n)(*[s.h.value for s in solvers]), n, (vp * n)(*[v.data_ptr() for v in vs]), ld,
            (vp * n)(*[x.data_ptr() for x in xs]), ld, (i64 * n)(*[v.shape[0] for v in vs]))
    return args, xs


def solve_grouped(solvers: list, vs: list, xs: list | None = None) -> list:
    """x_i = A_i^-1 v_i for factored solvers (``bem.Solver``, one device) in one persistent
    launch of FP64 Woodbury tiles (``bem_solve_batch``).  ``vs[i]`` is a complex128 tensor of
    shape (nrhs_i, N_i) on the device; ``xs`` (same shapes) receives the solutions and is
    allocated when None.  Runs on the first solver's stream, after every solver's earlier
    work; returns once it is done."""
    L = bem.load_library()
    args, xs = _grouped_args(solvers, vs, xs)
    st = L.bem_solve_batch(*args)
    if st != 0:
        raise bem.BemError(st, L.bem_last_error(solvers[0].h).decode())
    return xs


def grouped_stall_check(solvers: list, vs: list, stall_ms: int = 200) -> tuple[int, str]:
    """The failure-detection check of the grouped solve (``bem_solve_batch_stall_check``): the
    same launch with one completion counter that never reaches its target, so its waiting
    tiles give up after ``stall_ms``.  Returns (status, message); BEM_E_TIMEOUT (7) expected."""
    L = bem.load_library()
    args, _ = _grouped_args(solvers, vs, None)
    st = L.bem_solve_batch_stall_check(*args, int(stall_ms))
    return st, L.bem_last_error(solvers[0].h).decode()
