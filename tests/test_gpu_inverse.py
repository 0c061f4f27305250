"""The inverse-series solve (FTOEP_SOLVER_INVERSE: x = h_m * y with the whole inverse column
h_m = T_m^-1 e_1, one causal convolution of length 2 Np per mode pair) on the GPU, through
the C ABI, against the oracle, and against the half-split solve of the same plan set-up.

Cases: both kinds and the Crank-Nicolson kind, power-of-two and chirp-z sine sizes,
ragged N (the padding of the pair rows read as zero), four-step splits with n1 < n2 and
n1 = n2, nonzero u0 and phi, the scalar problem, double and mixed paths, host buffers,
batches where some problems take the inverse-series solve and the rest the half split
(chain and per-level schedules), the adjoint of double and mixed plans, and the rule that
takes the inverse series for the mixed sub-diffusion problems only
(FTOEP_SOLVER_INVERSE_MIXED_SUBDIFFUSION).  The library's own choice stays the half split
(test_library_choice_is_the_half_split).

Tolerances: the inverse-series solve rounds once over the whole time axis (one FFT of
length 2 Np), so its error is normwise -- about eps log2(2 Np) |h| |y| against the largest
values -- where the half split's follows each block's own values.  The sub-diffusion
inverse is positive and decaying and keeps the double error at 1e-12 of the data; the
hyperbolic inverse oscillates, and its double error is bounded here by 5e-12 of the data
(1.4e-12 measured at gamma 1.9, N = 70000); mixed 1e-6.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_1710_11593_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

INV = {"solver": 2}
HALF = {"solver": 1}


@pytest.fixture(scope="module")
def ft():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_11593_gb300 import ftoep
    ftoep.load()
    return ftoep


def _err(u, ref, *scales):
    s = max([np.max(np.abs(ref))] + [np.max(np.abs(x)) for x in scales if x is not None])
    d = np.asarray(u) - np.asarray(ref)
    return max(np.linalg.norm(d) / np.linalg.norm(ref), np.max(np.abs(d)) / s)


def _plan_solve(ft, specs, f, tuning, u0=None, phi=None, host=False):
    import torch
    if host:
        tf, t0, tp = np.ascontiguousarray(f), u0, phi
    else:
        tf = torch.from_numpy(np.ascontiguousarray(f)).cuda()
        t0 = None if u0 is None else torch.from_numpy(u0).cuda()
        tp = None if phi is None else torch.from_numpy(phi).cuda()
    with ft.Plan(specs, tuning) as plan:
        solvers = [plan.solver(i) for i in range(len(specs))]
        u = plan.solve(tf, u0=t0, phi=tp)
        plan.sync()
    return (u if host else u.cpu().numpy()), solvers


@pytest.mark.parametrize("kind,gamma,M,N,prec,init", [
    (0, 0.7, 31, 6000, 0, False),      # Np = 8192: n = 2^14 = 2^7 x 2^7
    (1, 1.5, 31, 9000, 1, True),       # mixed, Np = 16384: n1 = 2^7 < n2 = 2^8
    (2, 1.6, 40, 5000, 0, True),       # Crank-Nicolson kind, M+1 = 41 (chirp-z)
    (0, 0.3, 15, 20000, 1, False),     # mixed, Np = 32768
    (1, 1.9, 7, 70000, 0, True),       # Np = 131072: n = 2^18
    (0, 0.55, 100, 4500, 1, True),     # mixed, Np = 8192 just above one block, M+1 = 101
])
def test_inverse_vs_oracle(ft, oracle, kind, gamma, M, N, prec, init):
    rng = np.random.default_rng(N + M)
    f = rng.standard_normal((M, N))
    u0 = rng.standard_normal(M) if init else None
    phi = rng.standard_normal(M) if init and kind else None
    ref = oracle.march(kind, 1, gamma, f, u0=u0, phi=phi)
    u, solvers = _plan_solve(ft, [ft.ProblemSpec(kind, gamma, N, M, 1, prec)], f, INV, u0, phi)
    assert solvers == [ft.SOLVER_INVERSE]
    tol = (1e-12 if kind == 0 else 5e-12) if prec == 0 else 1e-6
    assert _err(u, ref, u0, phi) < tol


@pytest.mark.parametrize("prec", [0, 1])
def test_inverse_scalar_and_host_buffers(ft, oracle, prec):
    """No space (rows are independent scalar problems, lambda = 2), host buffers."""
    N, g, lam = 30000, 0.8, 2.0
    f = wl.random_field((6, N), seed=3)
    u0 = np.linspace(-1.0, 1.0, 6)
    ref = oracle.march(0, 0, g, f, lam=lam, u0=u0)
    u, solvers = _plan_solve(ft, [ft.ProblemSpec(0, g, N, 6, 0, prec, lam=lam)], f, INV, u0, None, host=True)
    assert solvers == [ft.SOLVER_INVERSE]
    assert _err(u, ref, u0) < (1e-12 if prec == 0 else 1e-6)


def test_small_problems_keep_the_half_split(ft):
    """One time block (N <= 4096), or 2 Np within the shared-memory convolution length: the
    block inverse already is the whole inverse, so the plan keeps the half-split solver."""
    with ft.Plan([ft.ProblemSpec(0, 0.5, 4096, 31, 1, 0), ft.ProblemSpec(1, 1.5, 3000, 15, 1, 1, ),
                  ft.ProblemSpec(0, 0.5, 4097, 31, 1, 0)], INV) as plan:
        assert [plan.solver(i) for i in range(3)] == [ft.SOLVER_HALFSPLIT, ft.SOLVER_HALFSPLIT,
                                                      ft.SOLVER_INVERSE]


def _modes_ref(oracle, f, kind, gamma, modes):
    M = f.shape[0]

    def one(m):
        fh = oracle.sine_project(f, m)
        return oracle.march_mode(kind, gamma, fh, oracle.mode_eigenvalue(m, M))
    with ThreadPoolExecutor(max_workers=len(modes)) as ex:
        return list(ex.map(one, modes))


@pytest.mark.parametrize("kind,gamma,prec", [(0, 0.6, 0), (1, 1.4, 1)])
def test_inverse_vs_half_split_long(ft, oracle, kind, gamma, prec):
    """M = 255, N = 40000 (Np = 65536): the two solvers agree (double 1e-12, mixed 1e-6 of
    each other), and three full-length sine modes of the inverse-series solution match the
    oracle's scalar march of each mode to that tolerance of the field's largest value (the
    unforced modes carry only the 1e-3 noise of the source)."""
    M, N = 255, 40000
    p = wl.config_diffusion(M=M, N=N, gamma=gamma) if kind == 0 else wl.config_wave(M=M, N=N, gamma=gamma)
    f = wl.materialize(p.source, p.kind, N, M) + 1e-3 * wl.random_field((M, N), seed=5)
    spec = [ft.ProblemSpec(kind, gamma, N, M, 1, prec)]
    ui, si = _plan_solve(ft, spec, f, INV)
    uh, sh = _plan_solve(ft, spec, f, HALF)
    assert si == [ft.SOLVER_INVERSE] and sh == [ft.SOLVER_HALFSPLIT]
    tol = 1e-12 if prec == 0 else 1e-6
    assert _err(ui, uh) < tol
    modes = [1, 3, 100]
    scale = np.max(np.abs(ui))
    for m, ref in zip(modes, _modes_ref(oracle, f, kind, gamma, modes)):
        assert np.max(np.abs(oracle.sine_project(ui, m) - ref)) < tol * scale, m


@pytest.mark.parametrize("sched", [1, 2])
def test_batch_mixing_solvers(ft, oracle, sched):
    """A batch asking for the inverse-series solve: problems of more than one block take it,
    the one-block ones keep the half split (on the chain schedule: the persistent kernel);
    double sub-diffusion, all against the oracle at 1e-12."""
    cases = [(0.7, 31, 20000), (0.4, 20, 3000), (0.5, 40, 9000), (0.6, 15, 4000), (0.9, 7, 50000)]
    specs = [ft.ProblemSpec(0, g, N, M, 1, 0) for g, M, N in cases]
    fs = [wl.random_field((M, N), seed=7 * i + 1) for i, (_, M, N) in enumerate(cases)]
    f = np.concatenate([x.reshape(-1) for x in fs])
    u, solvers = _plan_solve(ft, specs, f, {"scheduler": sched, "solver": 2})
    inv, half = ft.SOLVER_INVERSE, ft.SOLVER_HALFSPLIT
    assert solvers == [inv, half, inv, half, inv], solvers
    off = 0
    for (g, M, N), fi in zip(cases, fs):
        ui = u[off:off + M * N].reshape(M, N)
        off += M * N
        assert _err(ui, oracle.march(0, 1, g, fi)) < 1e-12, (g, M, N)


def test_library_choice_is_the_half_split(ft):
    with ft.Plan([ft.ProblemSpec(0, 0.5, 20000, 31, 1, 1), ft.ProblemSpec(1, 1.5, 20000, 31, 1, 0),
                  ft.ProblemSpec(0, 0.5, 20000, 31, 1, 0)]) as plan:
        assert [plan.solver(i) for i in range(3)] == [ft.SOLVER_HALFSPLIT] * 3


@pytest.mark.parametrize("prec", [0, 1])
def test_inverse_plan_adjoint(ft, oracle, prec):
    """Adjoint of an inverse-series plan: a double plan solves the transposed system with its
    double inverse spectra (1e-12), a mixed plan with the double half-split (its time sums
    and two blocks at N = 9000: 2.1e-12 measured, bound 5e-12)."""
    import torch
    M, N, g = 15, 9000, 0.65
    rng = np.random.default_rng(9)
    f = rng.standard_normal((M, N))
    gg = rng.standard_normal((M, N))
    with ft.Plan([ft.ProblemSpec(0, g, N, M, 1, prec)], INV) as plan:
        assert plan.solver(0) == ft.SOLVER_INVERSE
        u = plan.solve(torch.from_numpy(f).cuda())
        dldf, dg = plan.adjoint(torch.from_numpy(gg).cuda(), u)
        plan.sync()
        dldf = dldf.cpu().numpy()
    lam = oracle.adjoint_march(0, 1, g, gg)
    assert _err(dldf, lam) < (1e-12 if prec == 0 else 5e-12)
    ref = oracle.gamma_gradient(0, g, oracle.march(0, 1, g, f), lam)
    assert abs(dg[0] - ref) <= (1e-10 if prec == 0 else 1e-8) * abs(ref)


def test_mixed_subdiffusion_rule(ft, oracle):
    """FTOEP_SOLVER_INVERSE_MIXED_SUBDIFFUSION: the inverse series for the mixed sub-diffusion
    problems of more than one block, the half split for the hyperbolic, the double and the
    one-block ones; the mixed sub-diffusion solution matches the oracle at 1e-6 over the
    whole field and on its first 2048 levels against their own size."""
    import torch
    cases = [(0, 0.4, 15, 20000, 1), (1, 1.5, 15, 20000, 1), (0, 0.4, 15, 20000, 0), (0, 0.6, 15, 3000, 1)]
    specs = [ft.ProblemSpec(k, g, N, M, 1, pr) for k, g, M, N, pr in cases]
    with ft.Plan(specs, {"solver": ft.SOLVER_INVERSE_MIXED_SUBDIFFUSION}) as plan:
        assert [plan.solver(i) for i in range(4)] == [ft.SOLVER_INVERSE, ft.SOLVER_HALFSPLIT,
                                                      ft.SOLVER_HALFSPLIT, ft.SOLVER_HALFSPLIT]
    k, g, M, N, pr = cases[0]
    p = wl.config_diffusion(M=M, N=N, gamma=g)
    f = wl.materialize(p.source, p.kind, N, M) + 1e-3 * wl.random_field((M, N), seed=11)
    u, solvers = _plan_solve(ft, specs[:1], f, {"solver": ft.SOLVER_INVERSE_MIXED_SUBDIFFUSION})
    assert solvers == [ft.SOLVER_INVERSE]
    ref = oracle.march(0, 1, g, f)
    assert _err(u, ref) < 1e-6
    n0 = 2048
    d = u[:, :n0] - ref[:, :n0]
    assert np.linalg.norm(d) / np.linalg.norm(ref[:, :n0]) < 1e-6
