"""The Crank-Nicolson form of the hyperbolic scheme (FTOEP_L1_HYPERBOLIC_CN: the time terms
of Eq. 15 with the spatial operator averaged over levels n and n-1) on the GPU, through the
C ABI, against the oracle's march of the same scheme.

Sizes span several time blocks (small block tunings), the direct, shared-memory-FFT and
four-step levels, chirp-z sine sizes and ragged N, with nonzero u0 and phi; double path
1e-12 and mixed path 1e-6 (relative to the larger of |u|, |u0|, |phi|); the persistent chain
schedule in a batch mixed with the other kinds; the adjoint (the oracle's transposed march
and its gamma-gradient formula); and the O(tau^(3-g)) order of the scheme at N = 2^12..2^16.
"""
import math

import numpy as np
import pytest

from paper_1710_11593_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CN = 2
SMALL_TUNE = {"leaf": 8, "fft_tile": 64, "gemm_max_level": 16, "solver": 1}  # half-split


@pytest.fixture(scope="module")
def ft():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_11593_gb300 import ftoep
    ftoep.load()
    return ftoep


def _err(u, ref, *scales):
    """max(relative 2-norm error, max-abs error) against the data scale."""
    s = max([np.max(np.abs(ref))] + [np.max(np.abs(x)) for x in scales if x is not None])
    d = np.asarray(u) - np.asarray(ref)
    return max(np.linalg.norm(d) / np.linalg.norm(ref), np.max(np.abs(d)) / s)


def _solve(ft, specs, f, tuning=None, u0=None, phi=None):
    import torch
    tf = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    t0 = None if u0 is None else torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    tp = None if phi is None else torch.from_numpy(np.ascontiguousarray(phi)).cuda()
    with ft.Plan(specs, tuning) as plan:
        u = plan.solve(tf, u0=t0, phi=tp)
        plan.sync()
    return u.cpu().numpy()


@pytest.mark.parametrize("gamma,M,N,prec,tune", [
    (1.5, 31, 777, 0, SMALL_TUNE),                 # several blocks, every level kind
    (1.3, 40, 1500, 0, None),                      # M+1 = 41: chirp-z sine transform
    (1.8, 63, 3000, 1, {"fft_tile": 256}),         # mixed, 12 blocks
    (1.5, 100, 2000, 1, None),                     # mixed, M+1 = 101 (chirp-z)
    (1.95, 7, 9000, 0, {"fft_tile": 512, "solver": 1}),  # half-split four-step levels, ragged N
    (1.95, 7, 9000, 0, {"solver": 2}),             # inverse-series solve
    (1.4, 30, 12000, 1, {"solver": 2}),            # inverse-series solve, mixed
])
def test_cn_vs_oracle(ft, oracle, gamma, M, N, prec, tune):
    rng = np.random.default_rng(M * 7 + N)
    f = rng.standard_normal((M, N))
    u0 = rng.standard_normal(M)
    phi = rng.standard_normal(M)
    ref = oracle.march(CN, 1, gamma, f, u0=u0, phi=phi)
    u = _solve(ft, [ft.ProblemSpec(CN, gamma, N, M, 1, prec)], f, tune, u0, phi)
    tol = 1e-12 if prec == 0 else 1e-6
    assert _err(u, ref, u0, phi) < tol


@pytest.mark.parametrize("prec", [0, 1])
def test_cn_scalar(ft, oracle, prec):
    """D^g u = -lambda u + f (no space), lambda = 3, the average on the scalar term."""
    N, g, lam = 5000, 1.6, 3.0
    rng = np.random.default_rng(31)
    f = rng.standard_normal((4, N))
    u0 = rng.standard_normal(4)
    phi = rng.standard_normal(4)
    ref = oracle.march(CN, 0, g, f, lam=lam, u0=u0, phi=phi)
    u = _solve(ft, [ft.ProblemSpec(CN, g, N, 4, 0, prec, lam=lam)], f, None, u0, phi)
    assert _err(u, ref, u0, phi) < (1e-12 if prec == 0 else 1e-6)


@pytest.mark.parametrize("prec", [0, 1])
def test_cn_in_chain_batch(ft, oracle, prec):
    """A batch mixing the three kinds on the persistent chain schedule."""
    cases = [(CN, 1.5, 31, 5000), (1, 1.4, 20, 3000), (CN, 1.7, 64, 2500), (0, 0.6, 15, 7000)]
    specs = [ft.ProblemSpec(k, g, N, M, 1, prec) for k, g, M, N in cases]
    fs = [wl.random_field((M, N), seed=11 * i + M) for i, (_, _, M, N) in enumerate(cases)]
    f = np.concatenate([x.reshape(-1) for x in fs])
    u = _solve(ft, specs, f, {"scheduler": ft.SCHED_CHAIN, "solver": ft.SOLVER_HALFSPLIT})
    off = 0
    for (k, g, M, N), fi in zip(cases, fs):
        ref = oracle.march(k, 1, g, fi)
        ui = u[off:off + M * N].reshape(M, N)
        off += M * N
        assert _err(ui, ref) < (1e-12 if prec == 0 else 1e-6), (k, g, M, N)


def test_cn_adjoint(ft, oracle):
    """dL/df = A^-T g against the oracle's transposed march of the same scheme, and dL/dgamma
    against the oracle's gradient formula -<lam, (dT/dgamma) u> (the averaged spatial term
    does not depend on gamma)."""
    import torch
    M, N, g = 15, 400, 1.6
    rng = np.random.default_rng(4)
    f = rng.standard_normal((M, N))
    gg = rng.standard_normal((M, N))
    with ft.Plan([ft.ProblemSpec(CN, g, N, M, 1, 0)], SMALL_TUNE) as plan:
        tf = torch.from_numpy(f).cuda()
        u = plan.solve(tf)
        dldf, dg = plan.adjoint(torch.from_numpy(gg).cuda(), u)
        plan.sync()
        u, dldf = u.cpu().numpy(), dldf.cpu().numpy()
    uo = oracle.march(CN, 1, g, f)
    lam = oracle.adjoint_march(CN, 1, g, gg)
    assert _err(u, uo) < 1e-12
    assert _err(dldf, lam) < 1e-12
    ref = oracle.gamma_gradient(CN, g, uo, lam)
    assert abs(dg[0] - ref) <= 1e-10 * abs(ref)


def test_cn_order_on_gpu(ft):
    """u = t^3 sin(pi x_j) (the discrete sine eigenvector with its eigenvalue, so only the
    time error remains): the GPU solve converges at the order 3 - g of Eq. 15 (g = 1.5),
    where the kind with the spatial term at level n converges at first order."""
    M, g = 15, 1.5
    x = wl.space_points(M)
    sx = np.sin(np.pi * x)
    h = 1.0 / (M + 1)
    lam1 = 4.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    dc, dp = wl.caputo_power(3.0, g)
    errs = {CN: [], 1: []}
    for N in (4096, 16384, 65536):
        th = wl.time_points(1, N)
        t = wl.time_points(0, N)
        f = np.outer(sx, dc * th ** dp + lam1 * th ** 3)
        ex = np.outer(sx, t ** 3)
        for k in errs:
            u = _solve(ft, [ft.ProblemSpec(k, g, N, M, 1, 0)], f)
            errs[k].append(np.max(np.abs(u - ex)))
    r_cn = math.log2(errs[CN][-2] / errs[CN][-1]) / 2
    r_l = math.log2(errs[1][-2] / errs[1][-1]) / 2
    assert abs(r_cn - (3.0 - g)) < 0.06, errs
    assert abs(r_l - 1.0) < 0.1, errs
