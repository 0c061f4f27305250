"""Python binding of libftoep (C ABI in include/ftoep.h).

Argument marshalling only: every numerical step runs in the CUDA kernels of the
library.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays; their data
pointers are handed to the library, which detects host vs device memory.  If the
library has not been built, every entry point raises ``FtoepError`` -- there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libftoep.so")

FTOEP_OK, FTOEP_EINVAL, FTOEP_ENOMEM, FTOEP_ECUDA, FTOEP_ETIMEOUT, FTOEP_EUNSUPPORTED = range(6)
STATUS_NAMES = {0: "FTOEP_OK", 1: "FTOEP_EINVAL", 2: "FTOEP_ENOMEM", 3: "FTOEP_ECUDA", 4: "FTOEP_ETIMEOUT",
                5: "FTOEP_EUNSUPPORTED"}
L1_SUBDIFFUSION, L1_HYPERBOLIC, L1_HYPERBOLIC_CN = 0, 1, 2
SPACE_NONE, SPACE_DIRICHLET_LAPLACIAN = 0, 1
FP64, MIXED = 0, 1

SCHED_AUTO, SCHED_LEVELS, SCHED_CHAIN = 0, 1, 2
SOLVER_AUTO, SOLVER_HALFSPLIT, SOLVER_INVERSE, SOLVER_INVERSE_MIXED_SUBDIFFUSION = 0, 1, 2, 3

EXPORTS = ("ftoep_create", "ftoep_weights", "ftoep_solve", "ftoep_matvec", "ftoep_adjoint", "ftoep_profile",
           "ftoep_profile_read", "ftoep_matvec_noalloc", "ftoep_autotune", "ftoep_two_sided_cg", "ftoep_sync",
           "ftoep_last_error", "ftoep_destroy", "ftoep_problem_solver", "ftoep_gmres", "ftoep_advection_sweep")
K_BLOCK_SOLVE, K_CONV_SMEM, K_CONV_FOURSTEP, K_SINE, K_OTHER, K_RESIDUAL, K_CHAIN, K_INVERSE = range(8)
KERNEL_CLASSES = {K_BLOCK_SOLVE: "block_solve", K_CONV_SMEM: "conv_smem", K_CONV_FOURSTEP: "conv_fourstep",
                  K_SINE: "sine", K_OTHER: "other", K_RESIDUAL: "residual", K_CHAIN: "chain", K_INVERSE: "inverse"}


class FtoepError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class ftoep_problem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("space", ctypes.c_int), ("precision", ctypes.c_int),
                ("gamma", ctypes.c_double), ("T", ctypes.c_double), ("L", ctypes.c_double),
                ("lam", ctypes.c_double), ("N", ctypes.c_int64), ("M", ctypes.c_int64)]


class ftoep_tuning(ctypes.Structure):
    _fields_ = [("leaf", ctypes.c_int), ("fft_tile", ctypes.c_int), ("gemm_max_level", ctypes.c_int),
                ("scheduler", ctypes.c_int), ("streams", ctypes.c_int), ("solver", ctypes.c_int)]


_lib = None


def load(path: Optional[str] = None):
    """Load libftoep.so (built by ``paper_1710_11593_gb300.build``; FTOEP_LIB in the
    environment names another build of the same library)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = os.environ.get("FTOEP_LIB", LIB_PATH)
    if not os.path.exists(path):
        raise FtoepError(FTOEP_EUNSUPPORTED, f"{path} not found: build it with paper_1710_11593_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i64, ci, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    lib.ftoep_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ftoep_problem), ci,
                                 ctypes.POINTER(ftoep_tuning), vp]
    lib.ftoep_weights.argtypes = [vp, ci, dp, dp]
    lib.ftoep_solve.argtypes = [vp, dp, dp, dp, dp]
    lib.ftoep_matvec.argtypes = [vp, ci, dp, dp, i64, ci]
    lib.ftoep_adjoint.argtypes = [vp, dp, dp, dp, dp]
    lib.ftoep_profile.argtypes = [vp, ci]
    lib.ftoep_autotune.argtypes = [ctypes.POINTER(ftoep_problem), ci, vp, ctypes.POINTER(ftoep_tuning)]
    lib.ftoep_profile_read.argtypes = [vp, ci, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                       ctypes.POINTER(i64)]
    lib.ftoep_sync.argtypes = [vp]
    lib.ftoep_last_error.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.ftoep_destroy.argtypes = [vp]
    lib.ftoep_problem_solver.argtypes = [vp, ci, ctypes.POINTER(ci)]
    lib.ftoep_gmres.argtypes = [vp, ci, dp, dp, ci, ctypes.c_double, ci, ctypes.POINTER(ci),
                                ctypes.POINTER(ctypes.c_double)]
    lib.ftoep_advection_sweep.argtypes = [ci, ctypes.c_double, ctypes.c_double, ctypes.c_double, i64, i64, dp, dp,
                                          dp, dp, ci, vp]
    lib.ftoep_matvec_noalloc.argtypes = [vp, i64, vp, vp, i64, ci, vp]
    lib.ftoep_two_sided_cg.argtypes = [ctypes.c_double, ctypes.c_double, i64, dp, dp, ctypes.c_double, ci,
                                       ctypes.POINTER(ci), ctypes.POINTER(ctypes.c_double), vp]
    for name in EXPORTS:
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise FtoepError(FTOEP_EINVAL, "numpy arrays must be C-contiguous float64")
        return x.ctypes.data
    # torch tensor
    import torch
    if isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise FtoepError(FTOEP_EINVAL, "tensors must be contiguous float64")
        return x.data_ptr()
    raise FtoepError(FTOEP_EINVAL, f"unsupported array type {type(x)}")


def _numel(x) -> int:
    return int(x.size) if isinstance(x, np.ndarray) else int(x.numel())


def _last_error(plan_handle) -> str:
    buf = ctypes.create_string_buffer(512)
    load().ftoep_last_error(plan_handle, buf, 512)
    return buf.value.decode(errors="replace")


def _check(rc: int, plan_handle=None):
    if rc != FTOEP_OK:
        raise FtoepError(rc, _last_error(plan_handle))


def current_stream_handle() -> int:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


@dataclass
class ProblemSpec:
    kind: int
    gamma: float
    N: int
    M: int
    space: int = SPACE_DIRICHLET_LAPLACIAN
    precision: int = FP64
    T: float = 1.0
    L: float = 1.0
    lam: float = 1.0

    def to_c(self) -> ftoep_problem:
        return ftoep_problem(self.kind, self.space, self.precision, self.gamma, self.T, self.L, self.lam,
                             self.N, self.M)


def ftoep_create(problems: Sequence[ProblemSpec], tuning: Optional[dict] = None, stream: Optional[int] = None):
    """Create a plan (returns the opaque handle as an int)."""
    lib = load()
    arr = (ftoep_problem * len(problems))(*[p.to_c() for p in problems])
    tp = None
    if tuning:
        tp = ctypes.pointer(ftoep_tuning(int(tuning.get("leaf", 0)), int(tuning.get("fft_tile", 0)),
                                         int(tuning.get("gemm_max_level", 0)), int(tuning.get("scheduler", 0)),
                                         int(tuning.get("streams", 0)), int(tuning.get("solver", 0))))
    h = ctypes.c_void_p()
    st = current_stream_handle() if stream is None else stream
    rc = lib.ftoep_create(ctypes.byref(h), arr, len(problems), tp, ctypes.c_void_p(st))
    _check(rc, None)
    return h.value


def ftoep_weights(plan: int, iprob: int, a, dadgamma=None):
    _check(load().ftoep_weights(plan, iprob, _ptr(a), _ptr(dadgamma)), plan)


def ftoep_solve(plan: int, f, u, u0=None, phi=None):
    _check(load().ftoep_solve(plan, _ptr(f), _ptr(u), _ptr(u0), _ptr(phi)), plan)


def ftoep_matvec(plan: int, iprob: int, x, y, nlines: int, transpose: bool = False):
    _check(load().ftoep_matvec(plan, iprob, _ptr(x), _ptr(y), int(nlines), int(bool(transpose))), plan)


def ftoep_adjoint(plan: int, g, u, dldf, dldgamma=None):
    _check(load().ftoep_adjoint(plan, _ptr(g), _ptr(u), _ptr(dldf), _ptr(dldgamma)), plan)


def ftoep_profile(plan: int, enable: bool):
    _check(load().ftoep_profile(plan, int(bool(enable))), plan)


def ftoep_profile_read(plan: int, kclass: int):
    ms = ctypes.c_double()
    ops = ctypes.c_int64()
    nl = ctypes.c_int64()
    _check(load().ftoep_profile_read(plan, kclass, ctypes.byref(ms), ctypes.byref(ops), ctypes.byref(nl)), plan)
    return ms.value, ops.value, nl.value


def ftoep_matvec_noalloc(a, N: int, x, y, nlines: int, transpose: bool = False, stream: Optional[int] = None):
    """Allocation-free Toeplitz product (device pointers only, N <= 32768); see ftoep.h."""
    fn = load().ftoep_matvec_noalloc
    st = current_stream_handle() if stream is None else stream
    _check(fn(_ptr(a), int(N), _ptr(x), _ptr(y), int(nlines), int(bool(transpose)), ctypes.c_void_p(st)), None)


def two_sided_cg(f, gamma: float, T: float = 1.0, u=None, tol: float = 1e-12, maxit: int = 100000,
                 stream: Optional[int] = None):
    """Scheme 1 (two-sided ODE) by the fast conjugate gradient method (C ABI
    ftoep_two_sided_cg).  f: values at t_1 .. t_{N-1} (N = len(f) + 1), numpy or torch, host
    or device; u: initial guess (zeros if None), overwritten.  Returns (u, iterations,
    relative residual)."""
    n = _numel(f)
    if u is None:
        if isinstance(f, np.ndarray):
            u = np.zeros_like(f)
        else:
            import torch
            u = torch.zeros_like(f)
    it = ctypes.c_int()
    rr = ctypes.c_double()
    st = current_stream_handle() if stream is None else stream
    rc = load().ftoep_two_sided_cg(float(gamma), float(T), n + 1, _ptr(f), _ptr(u), float(tol), int(maxit),
                                   ctypes.byref(it), ctypes.byref(rr), ctypes.c_void_p(st))
    _check(rc, None)
    return u, it.value, rr.value


def ftoep_sync(plan: int):
    _check(load().ftoep_sync(plan), plan)


def ftoep_destroy(plan: int):
    load().ftoep_destroy(plan)


def ftoep_autotune(problems: Sequence[ProblemSpec], stream: Optional[int] = None) -> dict:
    """Time the candidate tunings (solver, block length, scheduler, internal streams) on the problems
    (C ABI ftoep_autotune) and return the fastest as a dict for Plan(..., tuning=...)."""
    lib = load()
    arr = (ftoep_problem * len(problems))(*[p.to_c() for p in problems])
    out = ftoep_tuning()
    st = current_stream_handle() if stream is None else stream
    rc = lib.ftoep_autotune(arr, len(problems), ctypes.c_void_p(st), ctypes.byref(out))
    _check(rc, None)
    return {"leaf": out.leaf, "fft_tile": out.fft_tile, "gemm_max_level": out.gemm_max_level,
            "scheduler": out.scheduler, "streams": out.streams, "solver": out.solver}


def tuning_key(problems: Sequence[ProblemSpec], device: str = "") -> str:
    """Cache key of a set of problems: the device name and the multiset of (N bucket, M
    bucket, precision, kind, space), buckets = ceil(log2) of N and of M+1."""
    import math
    sig = {}
    for p in problems:
        k = (math.ceil(math.log2(max(1, p.N))), math.ceil(math.log2(p.M + 1)), int(p.precision), int(p.kind),
             int(p.space))
        sig[k] = sig.get(k, 0) + 1
    items = ";".join(f"{a},{b},{c},{d},{e}x{n}" for (a, b, c, d, e), n in sorted(sig.items()))
    return f"{device}|{items}"


SHIPPED_TUNING = os.path.join(HERE, "tuned_gb300.json")
TUNING_FIELDS = ("leaf", "fft_tile", "gemm_max_level", "scheduler", "streams", "solver")


def _tuning_fields(entry: dict) -> dict:
    return {k: int(entry.get(k, 0)) for k in TUNING_FIELDS}


def tuning_cache_path() -> str:
    return os.environ.get("FTOEP_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "ftoep",
                                                               "tuning.json")


def autotune_cached(problems: Sequence[ProblemSpec], stream: Optional[int] = None, path: Optional[str] = None):
    """The autotuner's choice for these problems, from the JSON cache when a set of the same
    key (see tuning_key) was tuned on this device before, else from ftoep_autotune (stored
    in the cache).  Returns (tuning dict, True if it came from the cache)."""
    import json
    device = ""
    try:
        import torch
        if torch.cuda.is_available():
            device = torch.cuda.get_device_name()
    except Exception:
        pass
    key = tuning_key(problems, device)
    path = path or tuning_cache_path()
    cache = {}
    try:
        with open(path) as fh:
            cache = json.load(fh)
    except (OSError, ValueError):
        cache = {}
    if key in cache:
        return _tuning_fields(cache[key]), True
    try:  # the table shipped with the package (tune_table.py), read-only
        with open(SHIPPED_TUNING) as fh:
            shipped = json.load(fh)
        if key in shipped:
            return _tuning_fields(shipped[key]), True
    except (OSError, ValueError):
        pass
    tuning = ftoep_autotune(problems, stream)
    cache[key] = tuning
    try:
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass
    return tuning, False


class Plan:
    """Owning wrapper of an ftoep plan."""

    def __init__(self, problems: Sequence[ProblemSpec], tuning: Optional[dict] = None, stream: Optional[int] = None):
        self.problems = list(problems)
        self.handle = ftoep_create(self.problems, tuning, stream)
        self.total_field = sum(p.M * p.N for p in self.problems)
        self.total_vec = sum(p.M for p in self.problems)

    def close(self):
        if getattr(self, "handle", None):
            ftoep_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solver(self, iprob: int = 0) -> int:
        """SOLVER_HALFSPLIT or SOLVER_INVERSE: the solver the plan uses for problem iprob."""
        out = ctypes.c_int(0)
        _check(load().ftoep_problem_solver(self.handle, iprob, ctypes.byref(out)), self.handle)
        return out.value

    def gmres(self, f, u=None, iprob: int = 0, restart: int = 30, tol: float = 1e-12, maxit: int = 10000):
        """Restarted GMRES on problem iprob's space-time system (zero initial data), the
        comparison path of Sec. 3.2; u holds the initial guess (zeros if None).  Returns
        (u, Arnoldi steps, relative residual of u)."""
        N, M = self.problems[iprob].N, self.problems[iprob].M
        if _numel(f) != M * N:
            raise FtoepError(FTOEP_EINVAL, f"f has {_numel(f)} elements, problem expects {M * N}")
        if u is None:
            if isinstance(f, np.ndarray):
                u = np.zeros_like(f)
            else:
                import torch
                u = torch.zeros_like(f)
        it, rr = ctypes.c_int(0), ctypes.c_double(0.0)
        _check(load().ftoep_gmres(self.handle, iprob, _ptr(f), _ptr(u), restart, tol, maxit, ctypes.byref(it),
                                  ctypes.byref(rr)), self.handle)
        return u, it.value, rr.value

    def weights(self, iprob: int = 0, with_dgamma: bool = False):
        N = self.problems[iprob].N
        a = np.empty(N)
        d = np.empty(N) if with_dgamma else None
        ftoep_weights(self.handle, iprob, a, d)
        return (a, d) if with_dgamma else a

    def solve(self, f, u=None, u0=None, phi=None):
        if _numel(f) != self.total_field:
            raise FtoepError(FTOEP_EINVAL, f"f has {_numel(f)} elements, plan expects {self.total_field}")
        if u is None:
            if isinstance(f, np.ndarray):
                u = np.empty_like(f)
            else:
                import torch
                u = torch.empty_like(f)
        ftoep_solve(self.handle, f, u, u0, phi)
        return u

    def matvec(self, iprob: int, x, y=None, transpose: bool = False):
        N = self.problems[iprob].N
        n = _numel(x)
        if n % N:
            raise FtoepError(FTOEP_EINVAL, "x is not a whole number of lines")
        if y is None:
            if isinstance(x, np.ndarray):
                y = np.empty_like(x)
            else:
                import torch
                y = torch.empty_like(x)
        ftoep_matvec(self.handle, iprob, x, y, n // N, transpose)
        return y

    def adjoint(self, g, u=None, dldf=None, want_gamma: bool = True):
        if dldf is None:
            if isinstance(g, np.ndarray):
                dldf = np.empty_like(g)
            else:
                import torch
                dldf = torch.empty_like(g)
        dg = np.empty(len(self.problems)) if want_gamma else None
        ftoep_adjoint(self.handle, g, u, dldf, dg)
        return dldf, dg

    def sync(self):
        ftoep_sync(self.handle)

    def profile(self, enable: bool = True):
        ftoep_profile(self.handle, enable)

    def profile_read(self):
        """{class name: (event ms, timed operations, kernels launched)} since profile()."""
        return {name: ftoep_profile_read(self.handle, k) for k, name in KERNEL_CLASSES.items()}


def advection_sweep(scheme: int, f, gamma: float, T: float = 1.0, L: float = 1.0, u0=None, phi=None, u=None,
                    precision: int = FP64, stream: Optional[int] = None):
    """Schemes 2 and 3 of Sec. 3 (D^g u + u_x = f, inflow u(0, t) = 0) by the space-order sweep
    (C ABI ftoep_advection_sweep).  f: [M][N] (row i-1 = node x_i = i L/M); returns u."""
    M, N = (f.shape[0], f.shape[1]) if hasattr(f, "shape") and len(f.shape) == 2 else (1, _numel(f))
    if u is None:
        if isinstance(f, np.ndarray):
            u = np.empty_like(f)
        else:
            import torch
            u = torch.empty_like(f)
    st = current_stream_handle() if stream is None else stream
    rc = load().ftoep_advection_sweep(scheme, gamma, T, L, N, M, _ptr(f), _ptr(u0), _ptr(phi), _ptr(u), precision,
                                      ctypes.c_void_p(st))
    _check(rc, None)
    return u


def solve(f, gamma: float, kind: Optional[int] = None, precision: int = FP64, space: int = SPACE_DIRICHLET_LAPLACIAN,
          T: float = 1.0, L: float = 1.0, lam: float = 1.0, u0=None, phi=None, tuning: Optional[dict] = None):
    """One-shot solve of a single problem; f has shape [M, N] (time contiguous)."""
    if kind is None:
        kind = L1_SUBDIFFUSION if gamma < 1.0 else L1_HYPERBOLIC
    M, N = (1, f.shape[0]) if len(f.shape) == 1 else (f.shape[0], f.shape[1])
    with Plan([ProblemSpec(kind, gamma, N, M, space, precision, T, L, lam)], tuning) as p:
        u = p.solve(f, u0=u0, phi=phi)
        p.sync()
    return u
