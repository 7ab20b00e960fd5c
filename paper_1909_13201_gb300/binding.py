"""Thin Python binding of the C ABI in include/fsi.h (ctypes).

Argument marshalling only: every step of set-up and solve runs inside
libfsi.so (host set-up code and CUDA kernels).  PyTorch supplies device
memory and the CUDA stream.  There is no fallback: if the library is missing
or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

FSI_OK, FSI_ERR_ARG, FSI_ERR_CUDA, FSI_ERR_ALLOC, FSI_ERR_ZERO_PIVOT, FSI_ERR_NOT_CONVERGED, \
    FSI_ERR_BREAKDOWN, FSI_ERR_NONFINITE, FSI_ERR_STATE = range(9)
FSI_FP64, FSI_MIXED, FSI_MIXED_HALF = 0, 1, 2
FSI_FACTOR_AUTO, FSI_FACTOR_FP64, FSI_FACTOR_FP32, FSI_FACTOR_TF32 = 0, 1, 2, 3
FSI_SMOOTHER_FS, FSI_SMOOTHER_AS = 0, 1
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_ALLOC", 4: "ERR_ZERO_PIVOT",
                5: "ERR_NOT_CONVERGED", 6: "ERR_BREAKDOWN", 7: "ERR_NONFINITE", 8: "ERR_STATE"}

EXPORTED = ["fsi_setup_hierarchy", "fsi_setup_smoothers", "fsi_solve", "fsi_solve_batched",
            "fsi_adjoint", "fsi_get_sizes", "fsi_get_dof_map", "fsi_get_matrix", "fsi_get_transfer",
            "fsi_get_blocks", "fsi_apply_operator", "fsi_apply_smoother", "fsi_apply_vcycle",
            "fsi_setup_host_only", "fsi_get_pattern", "fsi_profile", "fsi_apply_smoother_noalloc",
            "fsi_get_cost", "fsi_autotune_layout",
            "fsi_autotune", "fsi_get_block_passes", "fsi_nl_setup", "fsi_nl_residual", "fsi_nl_inject",
            "fsi_nl_jacobian", "fsi_nl_step", "fsi_destroy", "fsi_last_error"]
FSI_NL_MAX_NEWTON = 32


class FSIError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Problem_t(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_fine", C.c_int), ("n_levels", C.c_int),
                ("material", C.POINTER(C.c_uint8)), ("advection", C.POINTER(C.c_double)),
                ("mu_s", C.c_double), ("lambda_s", C.c_double), ("rho_s", C.c_double),
                ("rho_f", C.c_double), ("mu_f", C.c_double), ("dt", C.c_double),
                ("bc_preset", C.c_int)]


class HierOpts_t(C.Structure):
    _fields_ = [("restriction", C.c_int), ("nonlinear", C.c_int)]


class NlParams_t(C.Structure):
    _fields_ = [("force", C.c_double), ("period", C.c_double), ("C1", C.c_double), ("C2", C.c_double)]


class NlOpts_t(C.Structure):
    _fields_ = [("nl_rtol", C.c_double), ("max_newton", C.c_int), ("lin_rtol", C.c_double),
                ("restart", C.c_int), ("max_iters", C.c_int)]


class NlStats_t(C.Structure):
    _fields_ = [("newton_steps", C.c_int), ("converged", C.c_int), ("status", C.c_int),
                ("lin_iterations", C.c_int * FSI_NL_MAX_NEWTON), ("lin_rho", C.c_double * FSI_NL_MAX_NEWTON),
                ("residual", C.c_double * (FSI_NL_MAX_NEWTON + 1)), ("jacobian_ms", C.c_double),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double), ("total_ms", C.c_double)]

    def to_dict(self):
        k = self.newton_steps
        return {"newton_steps": k, "converged": bool(self.converged), "status": self.status,
                "iterations": list(self.lin_iterations[:k]), "rho": list(self.lin_rho[:k]),
                "residuals": list(self.residual[:k + 1]), "jacobian_ms": self.jacobian_ms,
                "setup_ms": self.setup_ms, "solve_ms": self.solve_ms, "total_ms": self.total_ms}


class SmootherOpts_t(C.Structure):
    _fields_ = [("precision", C.c_int), ("patch", C.c_int), ("omega", C.c_double),
                ("nu_pre", C.c_int), ("nu_post", C.c_int), ("factor", C.c_int), ("variant", C.c_int),
                ("mult_levels", C.c_int), ("cascade", C.c_int)]


class SolveOpts_t(C.Structure):
    _fields_ = [("rtol", C.c_double), ("restart", C.c_int), ("max_iters", C.c_int),
                ("use_x0", C.c_int)]


class SolveStats_t(C.Structure):
    _fields_ = [("iterations", C.c_int), ("cycles", C.c_int), ("converged", C.c_int),
                ("status", C.c_int), ("r0", C.c_double), ("rN", C.c_double),
                ("rel_residual", C.c_double), ("rho", C.c_double), ("solve_ms", C.c_double)]

    def to_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = False) -> C.CDLL:
    """Load libfsi.so (optionally building it first).  Raises if absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise FileNotFoundError(f"{path} is missing: run __graft_entry__.build() first")
        _build.build()
    lib = C.CDLL(path)
    P, I, I64, I32, D, U8 = C.c_void_p, C.c_int, C.c_int64, C.c_int32, C.c_double, C.c_uint8
    lib.fsi_setup_hierarchy.argtypes = [C.POINTER(Problem_t), I, C.POINTER(HierOpts_t), P, C.POINTER(P)]
    lib.fsi_setup_smoothers.argtypes = [P, C.POINTER(SmootherOpts_t)]
    lib.fsi_solve.argtypes = [P, P, P, C.POINTER(SolveOpts_t), C.POINTER(SolveStats_t)]
    lib.fsi_solve_batched.argtypes = [P, C.POINTER(P), C.POINTER(P), C.POINTER(SolveOpts_t),
                                      C.POINTER(SolveStats_t)]
    lib.fsi_adjoint.argtypes = [P, P, P, P, P, C.POINTER(D), C.POINTER(SolveOpts_t), C.POINTER(SolveStats_t)]
    lib.fsi_get_sizes.argtypes = [P, I, I, C.POINTER(I64)]
    lib.fsi_get_dof_map.argtypes = [P, I, I, C.POINTER(I32), C.POINTER(I32), C.POINTER(I32)]
    lib.fsi_get_matrix.argtypes = [P, I, I, C.POINTER(I64), C.POINTER(I32), C.POINTER(D)]
    lib.fsi_get_transfer.argtypes = [P, I, I, I, C.POINTER(I64), C.POINTER(I32), C.POINTER(D)]
    lib.fsi_get_blocks.argtypes = [P, I, I, C.POINTER(I64), C.POINTER(I32)]
    lib.fsi_get_block_passes.argtypes = [P, I, I, C.POINTER(I32)]
    lib.fsi_apply_operator.argtypes = [P, I, I, P, P]
    lib.fsi_apply_smoother.argtypes = [P, I, I, P, P, I]
    lib.fsi_apply_vcycle.argtypes = [P, I, P, P, I]
    lib.fsi_setup_host_only.argtypes = [C.POINTER(Problem_t), C.POINTER(HierOpts_t), I, C.POINTER(P)]
    lib.fsi_get_pattern.argtypes = [P, I, I, C.POINTER(I64), C.POINTER(I32)]
    lib.fsi_profile.argtypes = [P, I, C.POINTER(D)]
    lib.fsi_apply_smoother_noalloc.argtypes = [P, I, I, P, P, I]
    lib.fsi_get_cost.argtypes = [P, I, C.POINTER(D)]
    lib.fsi_autotune_layout.argtypes = [P, C.POINTER(I), I, C.POINTER(SolveOpts_t), C.POINTER(I), C.POINTER(D)]
    lib.fsi_autotune.argtypes = [P, C.POINTER(I), I, C.POINTER(SolveOpts_t), C.POINTER(I), C.POINTER(D)]
    lib.fsi_nl_setup.argtypes = [P, C.POINTER(NlParams_t)]
    lib.fsi_nl_residual.argtypes = [P, I, I, P, P, D, P]
    lib.fsi_nl_inject.argtypes = [P, I, I, P, P]
    lib.fsi_nl_jacobian.argtypes = [P, I, P, P, D]
    lib.fsi_nl_step.argtypes = [P, I, P, P, D, C.POINTER(NlOpts_t), C.POINTER(NlStats_t)]
    lib.fsi_destroy.argtypes = [P]
    lib.fsi_destroy.restype = None
    lib.fsi_last_error.restype = C.c_char_p
    for name in EXPORTED:
        if name not in ("fsi_destroy", "fsi_last_error"):
            getattr(lib, name).restype = C.c_int
    _LIB = lib
    return lib


def _check(status, allow=()):
    if status != FSI_OK and status not in allow:
        raise FSIError(status, load_library().fsi_last_error().decode())
    return status


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _dptr(t) -> int:
    """Device pointer of a contiguous CUDA float64 tensor."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return t.data_ptr()


class FSISolver:
    """Handle on one fsi_ctx (one or many problems, same device and stream).

    host_only=True builds only the host-side structure (no GPU needed) for
    inspection: sizes, dof maps, patterns, transfers and block sets."""

    def __init__(self, problems, restriction: int = 0, stream=None, host_only=False, patch=None,
                 nonlinear: bool = False):
        lib = load_library()
        if not isinstance(problems, (list, tuple)):
            problems = [problems]
        self.problems = list(problems)
        self._keep = []
        arr = (Problem_t * len(problems))()
        for i, p in enumerate(problems):
            mat = np.ascontiguousarray(p.material, dtype=np.uint8)
            adv = np.ascontiguousarray(p.advection, dtype=np.float64)
            self._keep += [mat, adv]
            arr[i] = Problem_t(p.dim, p.n_fine, p.n_levels, _ptr(mat, C.c_uint8), _ptr(adv, C.c_double),
                               p.mu_s, p.lambda_s, p.rho_s, p.rho_f, p.mu_f, p.dt, p.bc_preset)
        self.ctx = C.c_void_p()
        ho = HierOpts_t(restriction, 1 if nonlinear else 0)
        if host_only:
            if len(problems) != 1:
                raise ValueError("host-only inspection takes one problem")
            b = problems[0].patch if patch is None else patch
            _check(lib.fsi_setup_host_only(arr, C.byref(ho), b, C.byref(self.ctx)))
            self.stream = None
        else:
            import torch
            self.stream = stream if stream is not None else torch.cuda.current_stream()
            _check(lib.fsi_setup_hierarchy(arr, len(problems), C.byref(ho), C.c_void_p(self.stream.cuda_stream),
                                           C.byref(self.ctx)))
        self._keep = []
        self.precision = None

    def __del__(self):
        try:
            if getattr(self, "ctx", None) and self.ctx.value:
                load_library().fsi_destroy(self.ctx)
                self.ctx = C.c_void_p()
        except Exception:
            pass

    def setup_smoothers(self, precision=FSI_FP64, patch=None, omega=None, nu_pre=1, nu_post=1,
                        factor=FSI_FACTOR_AUTO, variant=FSI_SMOOTHER_FS, mult_levels=0, cascade=False):
        """mult_levels: finest levels smoothed by the locally multiplicative
        sweep (0 = additive everywhere).  cascade: the swapped cascade (Krylov
        preconditioned by FS with a GMG V-cycle inside each field system)."""
        if patch is None:
            patch = self.problems[0].patch
        if omega is None:
            omega = getattr(self.problems[0], "omega", 1.0)
        so = SmootherOpts_t(precision, patch, omega, nu_pre, nu_post, factor, variant, mult_levels,
                            1 if cascade else 0)
        _check(load_library().fsi_setup_smoothers(self.ctx, C.byref(so)))
        self.precision = precision

    @staticmethod
    def _opts(rtol, restart, max_iters, use_x0):
        return SolveOpts_t(rtol, restart, max_iters, 1 if use_x0 else 0)

    def solve(self, b, x0=None, rtol=1e-8, restart=30, max_iters=1000, check=True, out=None):
        """Solve J2 x = b on problem 0 and return (x, stats).

        b: float64 tensor (CUDA; a host tensor is copied in and the result
        copied back).  x0: optional initial guess.  out: optional CUDA tensor
        that receives the solution (otherwise a new one is allocated)."""
        import torch
        host = not b.is_cuda
        bd = b.to("cuda", non_blocking=True) if host else b
        xd = out if out is not None else torch.empty_like(bd)
        use_x0 = x0 is not None
        if use_x0:
            xd.copy_(x0)
        st = SolveStats_t()
        opts = self._opts(rtol, restart, max_iters, use_x0)
        s = load_library().fsi_solve(self.ctx, _dptr(bd), _dptr(xd), C.byref(opts), C.byref(st))
        if check:
            _check(s)
        res = xd.to("cpu") if host else xd
        return res, st.to_dict()

    def solve_batched(self, bs, xs=None, rtol=1e-8, restart=30, max_iters=1000, check=True):
        import torch
        n = len(self.problems)
        xs = xs if xs is not None else [torch.empty_like(b) for b in bs]
        bp = (C.c_void_p * n)(*[_dptr(b) for b in bs])
        xp = (C.c_void_p * n)(*[_dptr(x) for x in xs])
        st = (SolveStats_t * n)()
        opts = self._opts(rtol, restart, max_iters, False)
        s = load_library().fsi_solve_batched(self.ctx, bp, xp, C.byref(opts), st)
        if check:
            _check(s)
        return xs, [st[i].to_dict() for i in range(n)]

    def adjoint(self, w, x, rtol=1e-8, restart=30, max_iters=1000, want_dA=True, want_dmu=True, check=True):
        import torch
        lam = torch.empty_like(w)
        nnz = self.sizes(self.n_levels - 1)["nnz"]
        dA = torch.empty(nnz, dtype=torch.float64, device=w.device) if want_dA else None
        dmu = C.c_double(0.0)
        st = SolveStats_t()
        opts = self._opts(rtol, restart, max_iters, False)
        s = load_library().fsi_adjoint(self.ctx, _dptr(w), _dptr(x), _dptr(lam),
                                       _dptr(dA) if want_dA else None,
                                       C.byref(dmu) if want_dmu else None, C.byref(opts), C.byref(st))
        if check:
            _check(s)
        return lam, dA, (dmu.value if want_dmu else None), st.to_dict()

    def autotune(self, candidates=(1, 2, 3), rtol=1e-8, restart=30, max_iters=300):
        """Per size class, time one solve per candidate Vanka group size and
        keep the fastest (fsi_autotune).  Returns (chosen[n_probs],
        times_ms[n_probs][n_cand])."""
        cand = (C.c_int * len(candidates))(*candidates)
        n = len(self.problems)
        chosen = (C.c_int * n)()
        times = np.zeros(n * len(candidates), np.float64)
        opts = self._opts(rtol, restart, max_iters, False)
        _check(load_library().fsi_autotune(self.ctx, cand, len(candidates), C.byref(opts), chosen,
                                           _ptr(times, C.c_double)))
        return list(chosen), times.reshape(n, len(candidates))

    def autotune_layout(self, lanes=(0, 1, 4), rtol=1e-8, restart=30, max_iters=300):
        """Lanes per row of the sparse copies (fsi_autotune_layout): times a
        solve of every problem at once per candidate and keeps the fastest.
        Returns (chosen, times_ms)."""
        cand = (C.c_int * len(lanes))(*lanes)
        chosen = C.c_int(0)
        times = np.zeros(len(lanes), np.float64)
        opts = self._opts(rtol, restart, max_iters, False)
        _check(load_library().fsi_autotune_layout(self.ctx, cand, len(lanes), C.byref(opts), C.byref(chosen),
                                                  _ptr(times, C.c_double)))
        return chosen.value, times.tolist()

    def profile(self, mode):
        """mode 1 start (reset), 0 stop, 2 read, 3 read and measure the
        float64 FMA rate.  Returns the counters of fsi_profile as a dict."""
        out = np.zeros(32, np.float64)
        _check(load_library().fsi_profile(self.ctx, mode, _ptr(out, C.c_double)))
        return {"smoother_launches": int(out[0]), "smoother_ms": out[1], "smoother_bytes": out[2],
                "spmv_launches": int(out[3]), "spmv_ms": out[4], "spmv_bytes": out[5],
                "kernel_launches": int(out[6]), "outer_launches": int(out[7]), "outer_ms": out[8],
                "outer_bytes": out[9], "outer_fma": out[10], "invert_launches": int(out[11]),
                "invert_ms": out[12], "invert_flops": out[13], "fine_blocks": int(out[14]),
                "restrict_launches": int(out[15]), "restrict_ms": out[16], "restrict_bytes": out[17],
                "prolong_launches": int(out[18]), "prolong_ms": out[19], "prolong_bytes": out[20],
                "fp64_gflops": out[21], "gs64_launches": int(out[22]), "gs64_ms": out[23], "gs64_fma": out[24],
                "gs1_launches": int(out[25]), "gs1_ms": out[26], "gs1_bytes": out[27], "gs64_bytes": out[28]}

    # ------------------------------------------------------------ nonlinear
    def nl_setup(self, force=20.0, period=1.0, C1=0.0, C2=0.0):
        """Prepare the nonlinear residual (fsi_nl_setup); needs nonlinear=True
        at construction.  C1 <= 0: C1 = mu_s / 3, C2 = C1 / 2."""
        _check(load_library().fsi_nl_setup(self.ctx, C.byref(NlParams_t(force, period, C1, C2))))

    def nl_residual(self, U, Un, t_new, level=None, prob=0):
        import torch
        level = self.n_levels - 1 if level is None else level
        R = torch.empty_like(U)
        _check(load_library().fsi_nl_residual(self.ctx, prob, level, _dptr(U), _dptr(Un), float(t_new), _dptr(R)))
        return R

    def nl_inject(self, U, level, prob=0):
        """State of level - 1 injected from the state U of level."""
        import torch
        n = self.sizes(level - 1, prob)["n"]
        Uc = torch.empty(n, dtype=torch.float64, device=U.device)
        _check(load_library().fsi_nl_inject(self.ctx, prob, level, _dptr(U), _dptr(Uc)))
        return Uc

    def nl_jacobian(self, U, Un, t_new, prob=0):
        """Replace the level operators by the Jacobians at U (fsi_nl_jacobian)."""
        _check(load_library().fsi_nl_jacobian(self.ctx, prob, _dptr(U), _dptr(Un), float(t_new)))
        self.precision = None

    def nl_step(self, Un, U, t_new, nl_rtol=1e-8, max_newton=10, lin_rtol=1e-8, restart=30, max_iters=1000,
                prob=0, check=True):
        """One Newton time step in place on U (initial guess in, new state out)."""
        st = NlStats_t()
        o = NlOpts_t(nl_rtol, max_newton, lin_rtol, restart, max_iters)
        s = load_library().fsi_nl_step(self.ctx, prob, _dptr(Un), _dptr(U), float(t_new), C.byref(o), C.byref(st))
        if check:
            _check(s)
        return st.to_dict()

    # ------------------------------------------------------------ accessors
    @property
    def n_levels(self):
        return self.problems[0].n_levels

    def sizes(self, level, prob=0):
        out = np.zeros(11, np.int64)
        _check(load_library().fsi_get_sizes(self.ctx, prob, level, _ptr(out, C.c_int64)))
        return {"n": int(out[0]), "nnz": int(out[1]), "n_blocks": int(out[2]), "max_block": int(out[3]),
                "offsets": out[4:11].copy()}

    def dof_map(self, level, prob=0):
        n = self.sizes(level, prob)["n"]
        f, c, nd = (np.zeros(n, np.int32) for _ in range(3))
        _check(load_library().fsi_get_dof_map(self.ctx, prob, level, _ptr(f, C.c_int32), _ptr(c, C.c_int32),
                                              _ptr(nd, C.c_int32)))
        return f, c, nd

    def matrix(self, level, prob=0):
        sz = self.sizes(level, prob)
        ptr = np.zeros(sz["n"] + 1, np.int64)
        col = np.zeros(sz["nnz"], np.int32)
        val = np.zeros(sz["nnz"], np.float64)
        _check(load_library().fsi_get_matrix(self.ctx, prob, level, _ptr(ptr, C.c_int64), _ptr(col, C.c_int32),
                                             _ptr(val, C.c_double)))
        return ptr, col, val

    def cost(self, prob=0):
        """Algorithmic bytes of one V-cycle, one float64 outer product, the
        Gram-Schmidt bytes per basis vector, and the fine unknowns
        (fsi_get_cost)."""
        out = (C.c_double * 4)()
        _check(load_library().fsi_get_cost(self.ctx, prob, out))
        return {"cycle_bytes": out[0], "outer_bytes": out[1], "gs_bytes_per_vector": out[2], "n": int(out[3])}

    def solve_bytes(self, iterations, restart=30, prob=0):
        """Algorithmic bytes of a solve of `iterations` Arnoldi steps:
        sum over steps j (mod restart) of cycle + outer + (j + 1) GS."""
        c = self.cost(prob)
        gs = sum((j % restart) + 1 for j in range(int(iterations)))
        return int(iterations) * (c["cycle_bytes"] + c["outer_bytes"]) + gs * c["gs_bytes_per_vector"]

    def operator_values(self, level=None, prob=0, device="cuda"):
        """The operator's values (CSR order of matrix()) as a float64 torch
        tensor: the differentiable stand-in for fsi_solve_autograd."""
        import torch
        level = self.n_levels - 1 if level is None else level
        _, _, val = self.matrix(level, prob)
        return torch.from_numpy(val).to(device)

    def pattern(self, level, prob=0):
        sz = self.sizes(level, prob)
        ptr = np.zeros(sz["n"] + 1, np.int64)
        col = np.zeros(sz["nnz"], np.int32)
        _check(load_library().fsi_get_pattern(self.ctx, prob, level, _ptr(ptr, C.c_int64), _ptr(col, C.c_int32)))
        return ptr, col

    def transfer(self, level, which, prob=0):
        lib = load_library()
        nrows = self.sizes(level, prob)["n"] if which == 0 else self.sizes(level - 1, prob)["n"]
        ptr = np.zeros(nrows + 1, np.int64)
        _check(lib.fsi_get_transfer(self.ctx, prob, level, which, _ptr(ptr, C.c_int64), None, None))
        col = np.zeros(int(ptr[-1]), np.int32)
        val = np.zeros(int(ptr[-1]), np.float64)
        _check(lib.fsi_get_transfer(self.ctx, prob, level, which, _ptr(ptr, C.c_int64), _ptr(col, C.c_int32),
                                    _ptr(val, C.c_double)))
        return ptr, col, val

    def blocks(self, level, prob=0):
        lib = load_library()
        nb = self.sizes(level, prob)["n_blocks"]
        ptr = np.zeros(nb + 1, np.int64)
        _check(lib.fsi_get_blocks(self.ctx, prob, level, _ptr(ptr, C.c_int64), None))
        idx = np.zeros(int(ptr[-1]), np.int32)
        _check(lib.fsi_get_blocks(self.ctx, prob, level, _ptr(ptr, C.c_int64), _ptr(idx, C.c_int32)))
        return ptr, idx

    def block_passes(self, level, prob=0):
        """Sweep pass (kind * k^dim + colour) of every field-split block, in block order."""
        nb = self.sizes(level, prob)["n_blocks"]
        out = np.zeros(nb, np.int32)
        _check(load_library().fsi_get_block_passes(self.ctx, prob, level, _ptr(out, C.c_int32)))
        return out

    def apply_operator(self, level, x, prob=0):
        import torch
        y = torch.empty_like(x)
        _check(load_library().fsi_apply_operator(self.ctx, prob, level, _dptr(x), _dptr(y)))
        return y

    def apply_smoother(self, level, r, transpose=False, prob=0):
        import torch
        y = torch.empty_like(r)
        _check(load_library().fsi_apply_smoother(self.ctx, prob, level, _dptr(r), _dptr(y), int(transpose)))
        return y

    def apply_smoother_noalloc(self, level, r, y, transpose=False, prob=0):
        """y = P2^{-1} r into the caller's CUDA tensor y, with no allocation by
        the library (working vectors in its static device array)."""
        _check(load_library().fsi_apply_smoother_noalloc(self.ctx, prob, level, _dptr(r), _dptr(y),
                                                          int(transpose)))
        return y

    def apply_vcycle(self, v, transpose=False, prob=0):
        import torch
        z = torch.empty_like(v)
        _check(load_library().fsi_apply_vcycle(self.ctx, prob, _dptr(v), _dptr(z), int(transpose)))
        return z


def _make_autograd():
    import torch

    class FSISolve(torch.autograd.Function):
        """x = J2^{-1} b with a hand-written backward: the adjoint solve
        J2^T lambda = dL/dx (transposed V-cycle preconditioner) gives
        dL/db = lambda, dL/dA_ij = -lambda_i x_j on the fine operator's
        sparsity pattern (CSR order of FSISolver.matrix) and
        dL/dmu_s = -lambda^T (dA/dmu_s) x, all from one fsi_adjoint call.

        `values` (the operator's nnz values) and `mu_s` (a 0-d tensor) are
        the differentiable stand-ins of the operator the solver was set up
        with: they must hold its values and shear modulus; the solve itself
        uses the library's assembled operator."""

        @staticmethod
        def forward(ctx, b, values, mu_s, solver, rtol=1e-8):
            x, st = solver.solve(b, rtol=rtol)
            ctx.solver = solver
            ctx.rtol = rtol
            ctx.save_for_backward(x)
            return x

        @staticmethod
        def backward(ctx, gx):
            (x,) = ctx.saved_tensors
            want_dA, want_dmu = ctx.needs_input_grad[1], ctx.needs_input_grad[2]
            lam, dA, dmu, _ = ctx.solver.adjoint(gx.contiguous(), x, rtol=ctx.rtol, want_dA=want_dA,
                                                 want_dmu=want_dmu)
            g_mu = torch.tensor(dmu, dtype=torch.float64, device=gx.device) if want_dmu else None
            return lam, dA if want_dA else None, g_mu, None, None

    return FSISolve


_FSISOLVE = None


def fsi_solve_autograd(b, solver, rtol=1e-8, values=None, mu_s=None):
    """Differentiable x = J2^{-1} b (torch.autograd.Function, adjoint backward).

    b: right-hand side (gradient dL/db = lambda).  values: optional tensor of
    the fine operator's nnz values in CSR order (see FSISolver.operator_values);
    its gradient is dL/dA on the pattern.  mu_s: optional 0-d float64 tensor
    holding the solid shear modulus of the problem; its gradient is dL/dmu_s."""
    import torch
    global _FSISOLVE
    if _FSISOLVE is None:
        _FSISOLVE = _make_autograd()
    nnz = solver.sizes(solver.n_levels - 1)["nnz"]
    if values is None:
        values = torch.zeros(nnz, dtype=torch.float64, device=b.device)
    elif values.numel() != nnz:
        raise ValueError(f"values must hold the fine operator's {nnz} entries")
    if mu_s is None:
        mu_s = torch.zeros((), dtype=torch.float64, device=b.device)
    return _FSISOLVE.apply(b, values, mu_s, solver, rtol)
