"""Thin ctypes binding of the C ABI in include/bem.h.

Argument marshalling only: every step of the solver runs in the CUDA library
``libbem_gb300.so`` (built by ``paper_2210_08580_gb300.build``).  PyTorch provides the
device memory and the stream.  If the library is missing the import of this module
succeeds but the first call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbem_gb300.so")

BEM_FP64 = 0
BEM_MIXED_BF16 = 1
BEM_OP_S, BEM_OP_W, BEM_OP_D = 1, 2, 4
MATS = {"S": 0, "W": 1, "N": 1, "D": 2, "B": 3, "U": 4, "Vh": 5, "sigma": 6, "Q": 7}
STATUS = {0: "BEM_OK", 1: "BEM_E_INVALID", 2: "BEM_E_NOMEM", 3: "BEM_E_CUDA", 4: "BEM_E_UNSUPPORTED",
          5: "BEM_E_SINGULAR", 6: "BEM_E_NOT_CONVERGED", 7: "BEM_E_TIMEOUT"}

# every symbol include/bem.h declares
EXPORTS = ("bem_default_options", "bem_create", "bem_destroy", "bem_last_error", "bem_set_stream",
           "bem_assemble", "filter_apply", "compress_compact", "factor", "bem_rhs_planewave",
           "solve_many", "solve_backward", "bem_get_matrix", "bem_get_info", "bem_timing_enable",
           "bem_timing_report", "solve_many_noalloc", "bem_farfield", "bem_farfield_adjoint",
           "bem_shape_vjp", "bem_rhs_pointsource", "bem_rhs_scale", "bem_amplitude_grad", "bem_shape_chain",
           "bem_assemble_batch", "bem_factor_rhs_planewave", "bem_solve_batch",
           "bem_solve_batch_stall_check")


class BemOptions(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("include_kernel_mode", ctypes.c_int),
                ("refine_rtol", ctypes.c_double), ("max_refine", ctypes.c_int),
                ("split_slices", ctypes.c_int), ("rhs_slices", ctypes.c_int), ("solve_slices", ctypes.c_int),
                ("filter_tile_n", ctypes.c_int), ("filter_split_k", ctypes.c_int), ("rhs_tile_n", ctypes.c_int),
                ("rhs_split_k", ctypes.c_int), ("asm_tile", ctypes.c_int)]


class BemInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("n", ctypes.c_int64), ("r", ctypes.c_int64),
                ("k", ctypes.c_double), ("h", ctypes.c_double), ("alpha", ctypes.c_double),
                ("beta", ctypes.c_double), ("sigma_max", ctypes.c_double), ("stage", ctypes.c_int),
                ("prec", ctypes.c_int), ("quad_points", ctypes.c_int64), ("equal_chord", ctypes.c_int),
                ("basis_block", ctypes.c_int), ("basis_iters", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class TorchDeviceMemory:
    """Device memory provider of a handle backed by PyTorch's caching allocator: blocks are
    taken on the handle's current stream (``stream_of()``), so a block the library hands back
    is reused only by work ordered after that stream's (what bem_create asks of a provider).
    ``allocated`` is the number of bytes currently held by the library.  ``fail_after`` (None:
    never) injects allocation failures for tests of the error paths: once that many more
    requests have been served, every request is refused (counted in ``refused``)."""

    def __init__(self, device: int, stream_of):
        self.device = device
        self.stream_of = stream_of
        self.sizes = {}
        self.allocated = 0
        self.peak = 0
        self.calls = 0
        self.fail_after = None
        self.refused = 0

        def _alloc(nbytes, _ctx):
            if self.fail_after is not None:
                if self.fail_after <= 0:
                    self.refused += 1
                    return None
                self.fail_after -= 1
            try:
                ptr = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream_of())
            except Exception:
                return None
            self.sizes[ptr] = int(nbytes)
            self.allocated += int(nbytes)
            self.peak = max(self.peak, self.allocated)
            self.calls += 1
            return ptr

        def _free(ptr, _ctx):
            if not ptr:
                return
            self.allocated -= self.sizes.pop(ptr, 0)
            try:
                torch.cuda.caching_allocator_delete(ptr)
            except Exception:       # interpreter shutdown: the allocator is gone already
                pass

        self.alloc_fn = ALLOC_FN(_alloc)        # kept alive as long as the provider
        self.free_fn = FREE_FN(_free)


class BemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build() "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(path)
    vp, i64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    L.bem_default_options.argtypes = [ctypes.POINTER(BemOptions)]
    L.bem_default_options.restype = None
    L.bem_create.argtypes = [ctypes.POINTER(vp), i32, vp, ctypes.POINTER(BemOptions), ALLOC_FN, FREE_FN, vp]
    L.bem_destroy.argtypes = [vp]
    L.bem_last_error.argtypes = [vp]
    L.bem_last_error.restype = ctypes.c_char_p
    L.bem_set_stream.argtypes = [vp, vp]
    L.bem_assemble.argtypes = [vp, vp, i64, dbl, ctypes.c_uint]
    L.filter_apply.argtypes = [vp, i64, dbl]
    L.compress_compact.argtypes = [vp, dbl, ctypes.POINTER(i64)]
    L.factor.argtypes = [vp]
    L.bem_rhs_planewave.argtypes = [vp, vp, i64, vp, vp, i64]
    L.bem_factor_rhs_planewave.argtypes = [vp, dbl, vp, i64, vp, vp, i64, ctypes.POINTER(i64)]
    L.bem_rhs_pointsource.argtypes = [vp, vp, i64, vp, vp, i64]
    L.solve_many.argtypes = [vp, vp, i64, vp, i64, i64, ctypes.POINTER(ctypes.c_int32),
                             ctypes.POINTER(ctypes.c_double)]
    L.solve_backward.argtypes = [vp, vp, i64, vp, i64, i64]
    L.bem_get_matrix.argtypes = [vp, i32, vp, i64]
    L.bem_get_info.argtypes = [vp, ctypes.POINTER(BemInfo)]
    L.solve_many_noalloc.argtypes = [vp, vp, i64, vp, i64, i64]
    L.solve_many_noalloc.restype = ctypes.c_int
    L.bem_farfield.argtypes = [vp, vp, i64, vp, i64, i64, vp, i64]
    L.bem_farfield_adjoint.argtypes = [vp, vp, i64, vp, i64, i64, vp, i64]
    L.bem_shape_vjp.argtypes = [vp, vp, vp, i64, vp, i64, vp, vp, vp, vp]
    L.bem_rhs_scale.argtypes = [vp, vp, i64, i64, vp, vp, i64]
    L.bem_amplitude_grad.argtypes = [vp, vp, i64, vp, i64, i64, vp]
    L.bem_shape_chain.argtypes = [vp, vp, i64, vp, vp]
    L.bem_assemble_batch.argtypes = [ctypes.POINTER(vp), i64, ctypes.POINTER(vp), ctypes.POINTER(i64),
                                     ctypes.POINTER(dbl)]
    L.bem_solve_batch.argtypes = [ctypes.POINTER(vp), i64, ctypes.POINTER(vp), ctypes.POINTER(i64),
                                  ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.bem_solve_batch_stall_check.argtypes = [ctypes.POINTER(vp), i64, ctypes.POINTER(vp), ctypes.POINTER(i64),
                                              ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.POINTER(i64), i32]
    L.bem_timing_enable.argtypes = [vp, i32]
    L.bem_timing_report.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    for name in ("bem_create", "bem_destroy", "bem_set_stream", "bem_assemble", "filter_apply",
                 "compress_compact", "factor", "bem_rhs_planewave", "bem_rhs_pointsource", "solve_many", "solve_backward",
                 "bem_get_matrix", "bem_get_info", "bem_timing_enable", "bem_timing_report", "bem_farfield",
                 "bem_farfield_adjoint", "bem_shape_vjp", "bem_rhs_scale", "bem_amplitude_grad", "bem_shape_chain",
                 "bem_assemble_batch", "bem_factor_rhs_planewave", "bem_solve_batch",
                 "bem_solve_batch_stall_check"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


class Solver:
    """One geometry, one handle: assemble -> filter_apply -> compress -> factor -> solve.

    Complex blocks of right-hand sides are torch.complex128 tensors of shape (nrhs, N)
    (column-major N x nrhs with leading dimension N on the C side).
    """

    def __init__(self, device: int = 0, prec: str = "fp64", include_kernel_mode: bool = True,
                 refine_rtol: float = 1e-10, max_refine: int = 6, stream: torch.cuda.Stream | None = None,
                 split_slices: int = 0, rhs_slices: int = 0, solve_slices: int = 0,
                 memory: str = "torch", tiles: dict | None = None):
        """memory: "torch" (default) -- every device buffer of the handle comes from
        PyTorch's caching allocator through the bem_create hooks; "cuda" -- the library
        allocates with the CUDA runtime itself.  tiles: optional tile shapes of the mixed
        path's products, {"filter_tile_n", "filter_split_k", "rhs_tile_n", "rhs_split_k"},
        and the assembly's vertex tile edge {"asm_tile": 15 | 23 | 31}."""
        self.L = load_library()
        self.device = torch.device("cuda", device)
        opt = BemOptions()
        self.L.bem_default_options(ctypes.byref(opt))
        opt.prec = BEM_MIXED_BF16 if prec == "mixed" else BEM_FP64
        opt.include_kernel_mode = 1 if include_kernel_mode else 0
        opt.refine_rtol = refine_rtol
        opt.max_refine = max_refine
        opt.split_slices = split_slices
        opt.rhs_slices = rhs_slices
        opt.solve_slices = solve_slices
        for key in ("filter_tile_n", "filter_split_k", "rhs_tile_n", "rhs_split_k", "asm_tile"):
            if tiles and key in tiles:
                setattr(opt, key, int(tiles[key]))
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        if memory == "torch":
            self.memory = TorchDeviceMemory(device, lambda: self.stream)
            hooks = (self.memory.alloc_fn, self.memory.free_fn, None)
        elif memory == "cuda":
            self.memory = None
            hooks = (ALLOC_FN(), FREE_FN(), None)
        else:
            raise ValueError("memory must be 'torch' or 'cuda'")
        self._check(self.L.bem_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream),
                                      ctypes.byref(opt), *hooks), None)
        self.h = h
        self.N = None
        self._ik = bool(include_kernel_mode)

    def _check(self, st, h=-1):
        if st != 0:
            hh = self.h if h == -1 else h
            msg = self.L.bem_last_error(hh).decode() if hh is not None else ""
            raise BemError(st, msg)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.bem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream: torch.cuda.Stream):
        """Enqueue later calls (and take later device memory) on ``stream``."""
        self.stream = stream
        self._check(self.L.bem_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)))

    # ---------------------------------------------------------------- stages
    def assemble(self, verts: torch.Tensor, k: float, ops: str = "SW"):
        v = verts.to(device=self.device, dtype=torch.float64).contiguous()
        assert v.ndim == 2 and v.shape[1] == 2
        mask = (BEM_OP_S if "S" in ops else 0) | (BEM_OP_W if ("W" in ops or "N" in ops) else 0) | \
               (BEM_OP_D if "D" in ops else 0)
        self._verts = v
        self._check(self.L.bem_assemble(self.h, _ptr(v), v.shape[0], float(k), mask))
        self.N = v.shape[0]
        self.k = float(k)

    def filter_apply(self, n_modes: int, alpha: float = 0.0):
        self._check(self.L.filter_apply(self.h, int(n_modes), float(alpha)))

    def compress(self, rel_tol: float) -> int:
        r = ctypes.c_int64()
        self._check(self.L.compress_compact(self.h, float(rel_tol), ctypes.byref(r)))
        return r.value

    def factor(self):
        self._check(self.L.factor(self.h))

    def factor_rhs_planewave(self, rel_tol: float, angles, out: torch.Tensor | None = None):
        """compress(rel_tol), factor() and rhs_planewave(angles) in one call, the right-hand
        sides overlapping the compression and the factor on a second stream; returns
        (rank, v)."""
        ang = torch.as_tensor(angles, dtype=torch.float64).to(self.device).contiguous()
        nrhs = ang.numel()
        v = out if out is not None else torch.empty((nrhs, self.N), dtype=torch.complex128, device=self.device)
        r = ctypes.c_int64()
        self._check(self.L.bem_factor_rhs_planewave(self.h, float(rel_tol), _ptr(ang), nrhs, None, _ptr(v), self.N,
                                                    ctypes.byref(r)))
        return r.value, v

    def rhs_planewave(self, angles, want_f: bool = False, want_v: bool = True):
        ang = torch.as_tensor(angles, dtype=torch.float64).to(self.device).contiguous()
        nrhs = ang.numel()
        f = torch.empty((nrhs, self.N), dtype=torch.complex128, device=self.device) if want_f else None
        v = torch.empty((nrhs, self.N), dtype=torch.complex128, device=self.device) if want_v else None
        self._check(self.L.bem_rhs_planewave(self.h, _ptr(ang), nrhs, _ptr(f) if f is not None else None,
                                             _ptr(v) if v is not None else None, self.N))
        return (f, v) if want_f else v

    def rhs_pointsource(self, sources, want_f: bool = False, want_v: bool = True):
        """Right-hand sides of line sources at ``sources`` ((nsrc, 2) positions off the curve)."""
        src = torch.as_tensor(sources, dtype=torch.float64).to(self.device).reshape(-1, 2).contiguous()
        nsrc = src.shape[0]
        f = torch.empty((nsrc, self.N), dtype=torch.complex128, device=self.device) if want_f else None
        v = torch.empty((nsrc, self.N), dtype=torch.complex128, device=self.device) if want_v else None
        self._check(self.L.bem_rhs_pointsource(self.h, _ptr(src), nsrc, _ptr(f) if f is not None else None,
                                               _ptr(v) if v is not None else None, self.N))
        return (f, v) if want_f else v

    def solve(self, v: torch.Tensor, report: bool = False, out: torch.Tensor | None = None):
        v = v.contiguous()
        nrhs = v.shape[0]
        x = out if out is not None else torch.empty_like(v)
        it = ctypes.c_int32(0)
        res = ctypes.c_double(0.0)
        self._check(self.L.solve_many(self.h, _ptr(v), self.N, _ptr(x), self.N, nrhs,
                                      ctypes.byref(it) if report else None,
                                      ctypes.byref(res) if report else None))
        if report:
            return x, it.value, res.value
        return x

    def solve_backward(self, g: torch.Tensor, out: torch.Tensor | None = None):
        g = g.contiguous()
        lam = out if out is not None else torch.empty_like(g)
        self._check(self.L.solve_backward(self.h, _ptr(g), self.N, _ptr(lam), self.N, g.shape[0]))
        return lam

    def farfield(self, obs_angles, x: torch.Tensor) -> torch.Tensor:
        """u_inf (nrhs, nobs) of the currents x (nrhs, N)."""
        obs = torch.as_tensor(obs_angles, dtype=torch.float64).to(self.device).contiguous()
        x = x.contiguous()
        out = torch.empty((x.shape[0], obs.numel()), dtype=torch.complex128, device=self.device)
        self._check(self.L.bem_farfield(self.h, _ptr(obs), obs.numel(), _ptr(x), self.N, x.shape[0],
                                        _ptr(out), obs.numel()))
        return out

    def farfield_adjoint(self, obs_angles, g: torch.Tensor) -> torch.Tensor:
        """F^H g (nrhs, N) for g (nrhs, nobs)."""
        obs = torch.as_tensor(obs_angles, dtype=torch.float64).to(self.device).contiguous()
        g = g.contiguous()
        out = torch.empty((g.shape[0], self.N), dtype=torch.complex128, device=self.device)
        self._check(self.L.bem_farfield_adjoint(self.h, _ptr(obs), obs.numel(), _ptr(g), obs.numel(), g.shape[0],
                                                _ptr(out), self.N))
        return out

    def shape_vjp(self, angles, amplitudes, obs_angles, x: torch.Tensor, gu: torch.Tensor,
                  lam: torch.Tensor) -> torch.Tensor:
        """d J / d verts (N, 2) for the misfit whose far-field gradient is gu (nrhs, nobs);
        x (nrhs, N) the solution, lam (nrhs, N) = A^-H F^H gu."""
        ang = torch.as_tensor(angles, dtype=torch.float64).to(self.device).contiguous()
        obs = torch.as_tensor(obs_angles, dtype=torch.float64).to(self.device).contiguous()
        amp = None if amplitudes is None else \
            torch.as_tensor(amplitudes, dtype=torch.complex128).to(self.device).contiguous()
        grad = torch.empty((self.N, 2), dtype=torch.float64, device=self.device)
        self._check(self.L.bem_shape_vjp(self.h, _ptr(ang), _ptr(amp) if amp is not None else None, ang.numel(),
                                         _ptr(obs), obs.numel(), _ptr(x.contiguous()), _ptr(gu.contiguous()),
                                         _ptr(lam.contiguous()), _ptr(grad)))
        return grad

    def rhs_scale(self, v: torch.Tensor, amplitudes) -> torch.Tensor:
        """a_w v_w for v (nrhs, N) and complex amplitudes (nrhs)."""
        v = v.contiguous()
        amp = torch.as_tensor(amplitudes, dtype=torch.complex128).to(self.device).contiguous()
        out = torch.empty_like(v)
        self._check(self.L.bem_rhs_scale(self.h, _ptr(v), self.N, v.shape[0], _ptr(amp), _ptr(out), self.N))
        return out

    def amplitude_grad(self, v: torch.Tensor, lam: torch.Tensor) -> torch.Tensor:
        """v_w^H lambda_w per right-hand side (nrhs complex)."""
        v, lam = v.contiguous(), lam.contiguous()
        g = torch.empty(v.shape[0], dtype=torch.complex128, device=self.device)
        self._check(self.L.bem_amplitude_grad(self.h, _ptr(v), self.N, _ptr(lam), self.N, v.shape[0], _ptr(g)))
        return g

    def shape_chain(self, tangent: torch.Tensor, grad_verts: torch.Tensor) -> torch.Tensor:
        """sum_{i,d} tangent[c, i, d] grad_verts[i, d] for tangent (ncoef, N, 2)."""
        t = tangent.to(device=self.device, dtype=torch.float64).contiguous()
        gv = grad_verts.to(device=self.device, dtype=torch.float64).contiguous()
        out = torch.empty(t.shape[0], dtype=torch.float64, device=self.device)
        self._check(self.L.bem_shape_chain(self.h, _ptr(t), t.shape[0], _ptr(gv), _ptr(out)))
        return out

    # ---------------------------------------------------------------- introspection
    def timing(self, enable: bool):
        self._check(self.L.bem_timing_enable(self.h, 1 if enable else 0))

    def timing_report(self) -> dict:
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        self._check(self.L.bem_timing_report(self.h, buf, len(buf)))
        return json.loads(buf.value.decode())

    def info(self) -> dict:
        inf = BemInfo()
        self._check(self.L.bem_get_info(self.h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in BemInfo._fields_}

    def matrix(self, name: str) -> torch.Tensor:
        """Copy of an internal matrix as a (rows, cols) complex128 tensor (``"Q"``, the real
        filter basis, as float64; ``"sigma"`` as a float64 vector)."""
        inf = self.info()
        N, r = inf["N"], inf["r"]
        nc = inf["n"] if self._include_kernel() else inf["n"] - 1
        which = MATS[name]
        if name == "sigma":
            out = torch.empty(nc, dtype=torch.float64, device=self.device)
            self._check(self.L.bem_get_matrix(self.h, which, _ptr(out), 0))
            torch.cuda.synchronize(self.device)
            return out
        if name == "Q":
            buf = torch.empty((nc, N), dtype=torch.float64, device=self.device)
            self._check(self.L.bem_get_matrix(self.h, which, _ptr(buf), N))
            torch.cuda.synchronize(self.device)
            return buf.T
        rows, cols = {"S": (N, N), "W": (N, N), "N": (N, N), "D": (N, N), "B": (nc, N),
                      "U": (N, r), "Vh": (r, N)}[name]
        buf = torch.empty((cols, rows), dtype=torch.complex128, device=self.device)
        self._check(self.L.bem_get_matrix(self.h, which, _ptr(buf), rows))
        torch.cuda.synchronize(self.device)
        return buf.T

    def _include_kernel(self) -> bool:
        return self._ik


def assemble_batch(solvers: list, verts_list: list, ks: list):
    """bem_assemble_batch: S and N of every solver's problem in one persistent launch (the
    solvers on one device; verts (N, 2) each, wavenumbers ks)."""
    L = load_library()
    n = len(solvers)
    vs = [v.to(device=solvers[i].device, dtype=torch.float64).contiguous() for i, v in enumerate(verts_list)]
    hs = (ctypes.c_void_p * n)(*[s.h.value for s in solvers])
    vp = (ctypes.c_void_p * n)(*[v.data_ptr() for v in vs])
    Ns = (ctypes.c_int64 * n)(*[v.shape[0] for v in vs])
    kk = (ctypes.c_double * n)(*[float(k) for k in ks])
    st = L.bem_assemble_batch(hs, n, vp, Ns, kk)
    if st != 0:
        raise BemError(st, L.bem_last_error(solvers[0].h).decode())
    for s, v, k in zip(solvers, vs, ks):
        s._verts = v
        s.N = v.shape[0]
        s.k = float(k)


class FarFieldSolve(torch.autograd.Function):
    """u_inf = F A^-1 v for a factored Solver (A = beta I + U V^H), differentiable in v.

    Forward: solve_many then bem_farfield.  Backward (complex-linear map, torch's
    conjugate-Wirtinger convention): grad_v = A^-H F^H grad_u, i.e. bem_farfield_adjoint then
    solve_backward -- the adjoint method, one extra solve per backward pass.  v: (nrhs, N)
    complex128 on the solver's device; returns (nrhs, nobs)."""

    @staticmethod
    def forward(ctx, v, solver, obs_angles):
        ctx.solver = solver
        ctx.obs = obs_angles
        x = solver.solve(v.detach())
        return solver.farfield(obs_angles, x)

    @staticmethod
    def backward(ctx, grad_u):
        s = ctx.solver
        g = s.farfield_adjoint(ctx.obs, grad_u.contiguous())
        return s.solve_backward(g), None, None


def farfield_solve(v: torch.Tensor, solver: "Solver", obs_angles) -> torch.Tensor:
    """Differentiable u_inf(v) (see FarFieldSolve)."""
    return FarFieldSolve.apply(v, solver, obs_angles)


class ShapeFarField(torch.autograd.Function):
    """u_inf (nrhs, nobs) of the star r(theta) = r0 + sum_m c_m cos(m theta) + s_m sin(m theta)
    on an equal-chord mesh of N vertices, for incident plane waves of angles ``angles`` with
    complex amplitudes ``amplitudes``; differentiable in the Fourier coefficients
    ``coef`` = (c_1..c_M, s_1..s_M) (float64) and in the amplitudes.

    Forward: mesh (host), bem_assemble .. factor (filter n_modes, no truncation), right-hand
    sides, bem_rhs_scale, solve_many, bem_farfield, on the FP64 or the mixed path (``prec``).
    Backward (adjoint method): lambda = solve_backward(bem_farfield_adjoint(gu)); the amplitude
    gradient from bem_amplitude_grad, d/dverts from bem_shape_vjp, chained to the coefficients
    by bem_shape_chain through the derivative of the equal-chord mesh
    (inputs.equal_chord_tangent)."""

    @staticmethod
    def forward(ctx, coef, amplitudes, r0, N, k, n_modes, angles, obs_angles, device=0, prec="fp64"):
        from . import inputs
        c = coef.detach().cpu().numpy()
        M = c.shape[0] // 2
        curve = inputs.PolarCurve(r0=float(r0), cos_coef=tuple(c[:M]), sin_coef=tuple(c[M:]))
        verts, theta, h = inputs.equal_chord_mesh(curve, int(N))
        s = Solver(device=device, prec=prec)
        dev = s.device
        s.assemble(torch.from_numpy(verts).to(dev), float(k), ops="SW")
        s.filter_apply(int(n_modes))
        s.compress(0.0)
        s.factor()
        ang = torch.as_tensor(angles, dtype=torch.float64).to(dev)
        obs = torch.as_tensor(obs_angles, dtype=torch.float64).to(dev)
        amp = amplitudes.detach().to(dev, torch.complex128)
        v0 = s.rhs_planewave(ang)
        x = s.solve(s.rhs_scale(v0, amp))
        u = s.farfield(obs, x)
        ctx.s, ctx.ang, ctx.obs, ctx.amp, ctx.v0, ctx.x = s, ang, obs, amp, v0, x
        ctx.tangent = torch.from_numpy(inputs.equal_chord_tangent(curve, theta, h))
        ctx.coef_device = coef.device
        return u

    @staticmethod
    def backward(ctx, gu):
        s = ctx.s
        gu = gu.contiguous()
        lam = s.solve_backward(s.farfield_adjoint(ctx.obs, gu))
        grad_a = s.amplitude_grad(ctx.v0, lam)
        gv = s.shape_vjp(ctx.ang, ctx.amp, ctx.obs, ctx.x, gu, lam)
        grad_c = s.shape_chain(ctx.tangent, gv).to(ctx.coef_device)
        s.close()
        return grad_c, grad_a, None, None, None, None, None, None, None, None


def shape_farfield(coef, amplitudes, r0, N, k, n_modes, angles, obs_angles, device=0, prec="fp64"):
    """Differentiable far field of a Fourier star (see ShapeFarField)."""
    return ShapeFarField.apply(coef, amplitudes, r0, N, k, n_modes, angles, obs_angles, device, prec)
