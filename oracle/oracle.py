"""Python face of the CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this module; the product path never imports it and shares no
code with it.  Every function here is a plain, slow, obviously-correct statement
of what the paper defines (Liu, Cheng, Li, Wang, arXiv 1710.11593):

* ``G``, ``Mk``: the L1 weights of Lemma 1 and the Sec. 3 definitions.
* ``time_coeffs``, ``scale``: the left-hand coefficients of Eq. 19/20 (kind 0) and of
  Eq. 17 (kind 1), first column of the lower-triangular Toeplitz time operator.
* ``march``: the direct time-marching procedure of Eq. 20 (and its hyperbolic and
  scalar analogues), O(M N^2), with a Thomas solve per level.  Kind 2 is the hyperbolic
  time discretization of Eq. 15 with the spatial term averaged over levels n and n-1
  (the Crank-Nicolson form of the scheme Eq. 15 is taken from).
* ``adjoint_march``: the transposed system, marched backwards.
* ``sine_project`` / ``march_mode``: one orthonormal sine mode, marched as a scalar
  problem with the mode's eigenvalue (used for sampled-mode checks).
* ``toeplitz_matvec``: a dense lower-triangular Toeplitz product (Sec. 3.1's A d).

The C part (oracle/oracle.c) is compiled by oracle/build.py.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None

SUBDIFFUSION = 0
HYPERBOLIC = 1
HYPERBOLIC_CN = 2
SPACE_NONE = 0
SPACE_DIRICHLET = 1

_dp = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64, dbl, cint = ctypes.c_int64, ctypes.c_double, ctypes.c_int
        lib.or_G.argtypes = [dbl, i64, _dp]
        lib.or_M.argtypes = [dbl, i64, _dp]
        lib.or_time_coeffs.argtypes = [cint, dbl, i64, _dp]
        lib.or_scale.argtypes = [cint, dbl, dbl]
        lib.or_scale.restype = dbl
        lib.or_time_coeffs_dgamma.argtypes = [cint, dbl, dbl, i64, _dp]
        lib.or_initial_weights.argtypes = [cint, dbl, dbl, i64, _dp, _dp]
        lib.or_march.argtypes = [cint, cint, dbl, dbl, dbl, dbl, i64, i64, _dp, _dp, _dp, _dp, cint]
        lib.or_adjoint_march.argtypes = [cint, cint, dbl, dbl, dbl, dbl, i64, i64, _dp, _dp, cint]
        lib.or_sine_project.argtypes = [i64, i64, _dp, i64, _dp]
        lib.or_toeplitz_matvec.argtypes = [_dp, i64, _dp, _dp, i64, cint]
        lib.or_advection_march.argtypes = [cint, dbl, dbl, dbl, i64, i64, _dp, _dp, _dp, _dp]
        for name in ("or_G", "or_M", "or_time_coeffs", "or_time_coeffs_dgamma", "or_initial_weights",
                     "or_march", "or_adjoint_march", "or_sine_project", "or_toeplitz_matvec",
                     "or_advection_march"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def default_threads() -> int:
    return os.cpu_count() or 1


def G(gamma: float, K: int) -> np.ndarray:
    """G_k = (k+1)^(1-g) - k^(1-g), k = 0..K-1 (Lemma 1), binary128 rounded to double."""
    out = np.empty(K)
    _check(_load().or_G(gamma, K, _ptr(out)), "G")
    return out


def Mk(gamma: float, K: int) -> np.ndarray:
    """M_k = (k+1)^(2-g) - k^(2-g), k = 0..K-1 (Sec. 3 definitions)."""
    out = np.empty(K)
    _check(_load().or_M(gamma, K, _ptr(out)), "M")
    return out


def time_coeffs(kind: int, gamma: float, N: int) -> np.ndarray:
    """Unscaled first column of the time operator (Eq. 4/19 for kind 0, Eq. 17 for kind 1)."""
    out = np.empty(N)
    _check(_load().or_time_coeffs(kind, gamma, N, _ptr(out)), "time_coeffs")
    return out


def scale(kind: int, gamma: float, tau: float) -> float:
    """mu = tau^-g/Gamma(2-g) (Lemma 2) or c = tau^-g/Gamma(3-g) (Eq. 17)."""
    return _load().or_scale(kind, gamma, tau)


def toeplitz_column(kind: int, gamma: float, N: int, T: float = 1.0) -> np.ndarray:
    """Full first column a_j = scale * coef_j of the time operator."""
    return scale(kind, gamma, T / N) * time_coeffs(kind, gamma, N)


def toeplitz_column_dgamma(kind: int, gamma: float, N: int, T: float = 1.0) -> np.ndarray:
    out = np.empty(N)
    _check(_load().or_time_coeffs_dgamma(kind, gamma, T / N, N, _ptr(out)), "time_coeffs_dgamma")
    return out


def initial_weights(kind: int, gamma: float, N: int, T: float = 1.0):
    wu0, wphi = np.empty(N), np.empty(N)
    _check(_load().or_initial_weights(kind, gamma, T / N, N, _ptr(wu0), _ptr(wphi)), "initial_weights")
    return wu0, wphi


def march(kind: int, space: int, gamma: float, f: np.ndarray, T: float = 1.0, L: float = 1.0,
          lam: float = 1.0, u0=None, phi=None, nthreads: int | None = None) -> np.ndarray:
    """Direct time marching (Eq. 20 and analogues).  f: [M][N] -> u: [M][N]."""
    f = _c64(f)
    if f.ndim == 1:
        f = f[None, :]
    M, N = f.shape
    u = np.zeros_like(f)
    u0 = None if u0 is None else _c64(u0)
    phi = None if phi is None else _c64(phi)
    rc = _load().or_march(kind, space, gamma, T, L, lam, N, M, _ptr(f), _ptr(u0), _ptr(phi), _ptr(u),
                          nthreads or default_threads())
    _check(rc, "march")
    return u


def adjoint_march(kind: int, space: int, gamma: float, g: np.ndarray, T: float = 1.0, L: float = 1.0,
                  lam: float = 1.0, nthreads: int | None = None) -> np.ndarray:
    """Solve A^T lam = g for the operator of ``march`` (backwards in time)."""
    g = _c64(g)
    if g.ndim == 1:
        g = g[None, :]
    M, N = g.shape
    out = np.zeros_like(g)
    rc = _load().or_adjoint_march(kind, space, gamma, T, L, lam, N, M, _ptr(g), _ptr(out),
                                  nthreads or default_threads())
    _check(rc, "adjoint_march")
    return out


def sine_project(f: np.ndarray, m: int) -> np.ndarray:
    """sqrt(2/(M+1)) * sum_j f_j^n sin(m pi j/(M+1)) for every time column n."""
    f = _c64(f)
    M, N = f.shape
    out = np.empty(N)
    _check(_load().or_sine_project(M, N, _ptr(f), m, _ptr(out)), "sine_project")
    return out


def mode_eigenvalue(m: int, M: int, L: float = 1.0) -> float:
    """Eigenvalue of the negative central second difference (-u_{j-1}+2u_j-u_{j+1})/h^2 with
    Dirichlet zeros for the sine vector sin(m pi j/(M+1)): (4/h^2) sin^2(m pi h/(2L))."""
    h = L / (M + 1)
    return 4.0 / (h * h) * math.sin(m * math.pi / (2 * (M + 1))) ** 2


def march_mode(kind: int, gamma: float, fhat: np.ndarray, lam_m: float, T: float = 1.0) -> np.ndarray:
    """Scalar march of one sine mode: D^g u = -lam_m u + fhat on the time grid."""
    return march(kind, SPACE_NONE, gamma, np.asarray(fhat)[None, :], T=T, lam=lam_m, nthreads=1)[0]


def toeplitz_matvec(a: np.ndarray, x: np.ndarray, transpose: bool = False) -> np.ndarray:
    """Dense lower-triangular Toeplitz product (first column a) on each row of x."""
    a = _c64(a)
    x = _c64(x)
    squeeze = x.ndim == 1
    if squeeze:
        x = x[None, :]
    n = x.shape[1]
    if a.shape[0] != n:
        raise ValueError("length mismatch")
    y = np.empty_like(x)
    _check(_load().or_toeplitz_matvec(_ptr(a), n, _ptr(x), _ptr(y), x.shape[0], int(bool(transpose))),
           "toeplitz_matvec")
    return y[0] if squeeze else y


def gamma_gradient(kind: int, gamma: float, u: np.ndarray, lam: np.ndarray, T: float = 1.0) -> float:
    """dL/dg = -sum over spatial lines of <lam_line, (dT/dg) u_line>, where T is the time
    operator, lam = A^-T dL/du and u = A^-1 f (f independent of g, zero initial data).
    dT/dg is the derivative of the first column, taken in binary128 (see oracle.c)."""
    u = _c64(u)
    lam = _c64(lam)
    N = u.shape[-1]
    da = toeplitz_column_dgamma(kind, gamma, N, T)
    return -float(np.sum(lam * toeplitz_matvec(da, u)))


# ----------------------------------------------------------------- Schemes 2 and 3 (advection)

def advection_march(scheme: int, gamma: float, f: np.ndarray, T: float = 1.0, L: float = 1.0, u0=None,
                    phi=None) -> np.ndarray:
    """Direct method of the advection schemes of Sec. 3 (time order, a forward sweep in
    space per level from u(0, t) = 0): scheme 2 (0 < g < 1, Eq. 12/13, the box scheme: L1 at
    x_{i-1/2} as the average of nodes i and i-1, f at (x_{i-1/2}, t_n)) and scheme 3
    (1 < g < 2, Eq. 16/17 with the upwind derivative at level n, f at (x_i, t_{n-1/2})).
    Nodes x_i = i L/M, i = 1..M.  f: [M][N] -> u: [M][N]."""
    f = _c64(f)
    M, N = f.shape
    u = np.zeros_like(f)
    u0 = None if u0 is None else _c64(u0)
    phi = None if phi is None else _c64(phi)
    rc = _load().or_advection_march(scheme, gamma, T, L, N, M, _ptr(f), _ptr(u0), _ptr(phi), _ptr(u))
    _check(rc, "advection_march")
    return u


# ----------------------------------------------------------------- Scheme 1 (two-sided ODE)

def two_sided_column(gamma: float, N: int, T: float = 1.0) -> np.ndarray:
    """First column of the symmetric Toeplitz matrix A of Scheme 1 (Eq. 7-9: the left L1
    formula of Eq. 4 plus the right one of Eq. 5, plus u, on u_1 .. u_{N-1} with
    u_0 = u_N = 0): a_0 = 1 + 2 mu G_0, a_d = mu (G_d - G_{d-1}) = mu W_d, d = 1 .. N-2,
    mu = tau^-g/Gamma(2-g).  G in binary128, rounded to double."""
    n = N - 1
    Gk = G(gamma, max(n, 1) + 1)
    mu = scale(0, gamma, T / N)
    a = np.empty(n)
    a[0] = 1.0 + 2.0 * mu * Gk[0]
    a[1:] = mu * (Gk[1:n] - Gk[0:n - 1])
    return a


def two_sided_matrix(gamma: float, N: int, T: float = 1.0) -> np.ndarray:
    """The dense (N-1) x (N-1) matrix A of Eq. 9."""
    a = two_sided_column(gamma, N, T)
    idx = np.arange(N - 1)
    return a[np.abs(idx[:, None] - idx[None, :])]


def two_sided_solve(gamma: float, f: np.ndarray, T: float = 1.0) -> np.ndarray:
    """u = A^-1 f for Scheme 1 by Gaussian elimination on the dense matrix (the paper's
    "Gauss method"), f = (f_1 .. f_{N-1})."""
    f = _c64(f)
    return np.linalg.solve(two_sided_matrix(gamma, f.shape[0] + 1, T), f)
