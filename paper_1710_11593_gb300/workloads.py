"""Seeded synthetic workloads: source terms, exact solutions and problem tables.

This module holds input generation only -- no step of the numerical method.  It is
shared by the tests, the benchmark and the CPU baseline so that all of them see the
same inputs.  Every field is a finite sum of separable terms

    f(x, t) = sum_i  c_i * t^{p_i} * sin(k_i * pi * x / L)       (k_i = 0: no x-factor)

sampled on x_j = j*h (j = 1..M, h = L/(M+1)) and on the time levels of the scheme:
t_n = n*tau for the sub-diffusion scheme (Eq. 19) and t_{n-1/2} = (n-1/2)*tau for the
hyperbolic scheme (Eq. 15/17), n = 1..N, tau = T/N.

Manufactured solutions use D^g t^p = Gamma(p+1)/Gamma(p+1-g) t^{p-g} (Caputo
derivative, Eq. 1, of a power with p > g-ish regularity) and (sin k pi x)'' =
-(k pi)^2 sin k pi x.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

SUBDIFFUSION = 0
HYPERBOLIC = 1
SPACE_NONE = 0
SPACE_DIRICHLET = 1

Term = Tuple[float, float, int]  # (coefficient, power of t, sine wavenumber k; 0 = none)


@dataclass
class Problem:
    kind: int
    space: int
    gamma: float
    N: int
    M: int
    T: float = 1.0
    L: float = 1.0
    lam: float = 1.0          # scalar problems only: D^g u = -lam*u + f
    source: List[Term] = field(default_factory=list)
    exact: Optional[List[Term]] = None

    @property
    def unknowns(self) -> int:
        return self.M * self.N


def caputo_power(p: float, g: float) -> Tuple[float, float]:
    """D^g t^p = coef * t^(p-g): returns (coef, p-g)."""
    return math.gamma(p + 1.0) / math.gamma(p + 1.0 - g), p - g


def time_points(kind: int, N: int, T: float = 1.0) -> np.ndarray:
    tau = T / N
    n = np.arange(1, N + 1, dtype=np.float64)
    return n * tau if kind == SUBDIFFUSION else (n - 0.5) * tau


def space_points(M: int, L: float = 1.0) -> np.ndarray:
    h = L / (M + 1)
    return np.arange(1, M + 1, dtype=np.float64) * h


def materialize(terms: Sequence[Term], kind: int, N: int, M: int, T: float = 1.0, L: float = 1.0,
                t: Optional[np.ndarray] = None, dtype=np.float64) -> np.ndarray:
    """Evaluate sum_i c_i t^p_i sin(k_i pi x/L) on the grid -> array [M][N] (numpy)."""
    if t is None:
        t = time_points(kind, N, T)
    x = space_points(M, L)
    out = np.zeros((M, len(t)), dtype=np.float64)
    for c, p, k in terms:
        tt = c * np.power(t, p)
        sx = np.ones(M) if k == 0 else np.sin(k * math.pi * x / L)
        out += np.outer(sx, tt)
    return out.astype(dtype, copy=False)


def materialize_torch(terms: Sequence[Term], kind: int, N: int, M: int, T: float = 1.0, L: float = 1.0,
                      device="cuda", out=None):
    """Same as ``materialize`` but built on a torch device (outer products, float64)."""
    import torch
    tau = T / N
    n = torch.arange(1, N + 1, dtype=torch.float64, device=device)
    t = n * tau if kind == SUBDIFFUSION else (n - 0.5) * tau
    x = torch.arange(1, M + 1, dtype=torch.float64, device=device) * (L / (M + 1))
    if out is None:
        out = torch.zeros((M, N), dtype=torch.float64, device=device)
    else:
        out.zero_()
    for c, p, k in terms:
        tt = c * torch.pow(t, p)
        sx = torch.ones(M, dtype=torch.float64, device=device) if k == 0 else torch.sin(k * math.pi * x / L)
        out.addr_(sx, tt)
    return out


def manufactured_source(exact: Sequence[Term], g: float, space: int, lam: float = 1.0, L: float = 1.0) -> List[Term]:
    """Source f with D^g u - u_xx = f (space=1) or D^g u + lam*u = f (space=0) for the
    exact solution u = sum c t^p sin(k pi x/L)."""
    src: List[Term] = []
    for c, p, k in exact:
        dc, dp = caputo_power(p, g)
        src.append((c * dc, dp, k))
        if space == SPACE_DIRICHLET:
            src.append((c * (k * math.pi / L) ** 2, p, k))
        else:
            src.append((c * lam, p, k))
    return src


# --------------------------------------------------------------------------- configs

def config_scalar(N: int = 1024, gamma: float = 0.5) -> Problem:
    """D^g u = -u + f on [0,1], exact u = t^2 (f = 2 t^(2-g)/Gamma(3-g) + t^2)."""
    exact = [(1.0, 2.0, 0)]
    return Problem(SUBDIFFUSION, SPACE_NONE, gamma, N, 1, lam=1.0,
                   source=manufactured_source(exact, gamma, SPACE_NONE, lam=1.0), exact=exact)


def config_diffusion(M: int = 1023, N: int = 65536, gamma: float = 0.7) -> Problem:
    """D^g u = u_xx + f on (0,1)x(0,1], Dirichlet zeros, exact u = t^2 sin(pi x)."""
    exact = [(1.0, 2.0, 1)]
    return Problem(SUBDIFFUSION, SPACE_DIRICHLET, gamma, N, M,
                   source=manufactured_source(exact, gamma, SPACE_DIRICHLET), exact=exact)


def config_table9(h_inv: int, gamma: float) -> Problem:
    """Example 4 of the paper: exact u = t^3 sin(pi x), h = tau = 1/h_inv."""
    exact = [(1.0, 3.0, 1)]
    return Problem(SUBDIFFUSION, SPACE_DIRICHLET, gamma, h_inv, h_inv - 1,
                   source=manufactured_source(exact, gamma, SPACE_DIRICHLET), exact=exact)


def config_wave(M: int = 4095, N: int = 262144, gamma: float = 1.5) -> Problem:
    """Hyperbolic 1<g<2 with u(x,0)=u_t(x,0)=0, exact u = t^3 sin(pi x) + t^3 sin(3 pi x)/9,
    f sampled at t_{n-1/2}."""
    exact = [(1.0, 3.0, 1), (1.0 / 9.0, 3.0, 3)]
    return Problem(HYPERBOLIC, SPACE_DIRICHLET, gamma, N, M,
                   source=manufactured_source(exact, gamma, SPACE_DIRICHLET), exact=exact)


def config_adjoint(M: int = 1023, N: int = 65536, gamma: float = 0.6) -> Problem:
    """Differentiation workload: the config-2 type source at g = 0.6 (exact u = t^2 sin pi x
    at that order).  The observation u_obs is produced at g = 0.55 by the caller."""
    exact = [(1.0, 2.0, 1)]
    return Problem(SUBDIFFUSION, SPACE_DIRICHLET, gamma, N, M,
                   source=manufactured_source(exact, gamma, SPACE_DIRICHLET), exact=exact)


def config_batched(nprob: int = 512, seed: int = 1234, n_range=(2 ** 10, 2 ** 17), m_range=(63, 2047),
                   g_sub=(0.1, 0.95), g_hyp=(1.05, 1.9), nterms: int = 4) -> List[Problem]:
    """Ragged batch: N and M integer log-uniform, g uniform on (0.1,0.95) u (1.05,1.9)
    (branch chosen with probability proportional to its length), source = sum of 4 terms
    A t^p sin(k pi x) with A ~ N(0,1), p ~ U[1,3], k ~ U{1..8}."""
    rng = np.random.default_rng(seed)
    probs = []
    len_sub = g_sub[1] - g_sub[0]
    len_hyp = g_hyp[1] - g_hyp[0]
    for _ in range(nprob):
        N = int(round(math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))))
        M = int(round(math.exp(rng.uniform(math.log(m_range[0]), math.log(m_range[1])))))
        if rng.uniform() < len_sub / (len_sub + len_hyp):
            kind, g = SUBDIFFUSION, float(rng.uniform(*g_sub))
        else:
            kind, g = HYPERBOLIC, float(rng.uniform(*g_hyp))
        terms = []
        for _ in range(nterms):
            A = float(rng.standard_normal())
            p = float(rng.uniform(1.0, 3.0))
            k = int(rng.integers(1, 9))
            terms.append((A, p, k))
        probs.append(Problem(kind, SPACE_DIRICHLET, g, N, M, source=terms))
    return probs


def two_sided_example1(N: int, gamma: float):
    """Example 1 of the paper (two-sided ODE, Eq. 2 on (0,1), u(0) = u(1) = 0), exact
    u = t(1-t) on the interior grid t_n = n/N, n = 1 .. N-1, and its source
    f = D_left^g u + D_right^g u + u.  Both Caputo derivatives in closed form:
    D_left^g (t - t^2) = L(t) with L(s) = s^(1-g)/Gamma(2-g) - 2 s^(2-g)/Gamma(3-g), and the
    right derivative (Eq. 6) is the left one of the reflected function, L(1-t).
    Returns (t, f, u)."""
    t = np.arange(1, N, dtype=np.float64) / N
    L = lambda s: s ** (1 - gamma) / math.gamma(2 - gamma) - 2 * s ** (2 - gamma) / math.gamma(3 - gamma)
    u = t * (1 - t)
    return t, L(t) + L(1 - t) + u, u


def noise(shape, sigma: float, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape) * sigma


def random_field(shape, seed: int, dtype=np.float64) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)
