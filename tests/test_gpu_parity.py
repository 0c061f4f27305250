"""GPU parity: libftoep (through its C ABI) against the CPU oracle, element by element.

Sizes are small enough for the O(M N^2) oracle but span several time blocks, the
direct, shared-memory-FFT and four-step convolution levels, ragged tails (N not a power
of two, odd M) and both schemes.  Tolerances: double path 1e-12 relative (2-norm and
max-abs over max |u|); mixed path 1e-6 relative.
"""
import numpy as np
import pytest

from paper_1710_11593_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _rel(u, ref):
    u = np.asarray(u)
    ref = np.asarray(ref)
    l2 = np.linalg.norm(u - ref) / np.linalg.norm(ref)
    mx = np.max(np.abs(u - ref)) / np.max(np.abs(ref))
    return max(l2, mx)


@pytest.fixture(scope="module")
def ft():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_11593_gb300 import ftoep
    ftoep.load()
    return ftoep


def _solve_gpu(ft, kind, gamma, f, space=1, precision=0, lam=1.0, u0=None, phi=None, tuning=None):
    import torch
    M, N = f.shape
    ft_f = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    t_u0 = None if u0 is None else torch.from_numpy(u0).cuda()
    t_phi = None if phi is None else torch.from_numpy(phi).cuda()
    with ft.Plan([ft.ProblemSpec(kind, gamma, N, M, space, precision, lam=lam)], tuning) as plan:
        u = plan.solve(ft_f, u0=t_u0, phi=t_phi)
        plan.sync()
    return u.cpu().numpy()


SMALL_TUNE = {"leaf": 8, "fft_tile": 64, "gemm_max_level": 16, "solver": 1}  # half-split


def test_config1_scalar(ft, oracle):
    """Config 1: D^0.5 u = -u + f, N = 1024, exact u = t^2."""
    p = wl.config_scalar()
    f = wl.materialize(p.source, p.kind, p.N, 1)
    ref = oracle.march(p.kind, p.space, p.gamma, f, lam=1.0)
    u = _solve_gpu(ft, p.kind, p.gamma, f, space=0, lam=1.0)
    assert _rel(u, ref) < 1e-12
    ex = wl.materialize(p.exact, p.kind, p.N, 1)
    assert np.max(np.abs(u - ex)) < 2.0 * (1.0 / p.N) ** 1.5


@pytest.mark.parametrize("kind,gamma,M,N,tune", [
    (0, 0.7, 31, 600, None),
    (0, 0.7, 31, 600, SMALL_TUNE),
    (0, 0.3, 15, 1000, {"leaf": 4, "fft_tile": 32, "gemm_max_level": 4, "solver": 1}),
    (1, 1.5, 31, 777, SMALL_TUNE),
    (1, 1.9, 63, 300, None),
    (0, 0.95, 7, 2049, {"leaf": 16, "fft_tile": 128, "gemm_max_level": 32, "solver": 1}),
])
def test_fp64_random_rhs(ft, oracle, kind, gamma, M, N, tune):
    f = wl.random_field((M, N), seed=M * 1000 + N)
    ref = oracle.march(kind, 1, gamma, f)
    u = _solve_gpu(ft, kind, gamma, f, tuning=tune)
    assert _rel(u, ref) < 1e-12


@pytest.mark.parametrize("kind,gamma,M,N,prec", [
    (0, 0.7, 100, 700, 0),    # M+1 = 101 (prime): chirp-z sine transform
    (1, 1.5, 62, 500, 0),     # M+1 = 63
    (0, 0.4, 2, 300, 0),      # M+1 = 3, smallest odd size
    (0, 0.8, 200, 1200, 1),   # mixed, M+1 = 201
    (1, 1.8, 2046, 150, 1),   # mixed, M+1 = 2047 = 23*89, P = 8192
    # float chirp-z, a convolution minus a correlation of length P >= 2K - 3 (K = M+1)
    (0, 0.6, 40, 900, 1),     # mixed, K = 41: P = 128
    (1, 1.3, 682, 300, 1),    # mixed, K = 683: P = 2048
    (0, 0.5, 1024, 200, 1),   # mixed, K = 1025: 2K - 3 = P - 1, the input fills [0, P/2)
    (1, 1.4, 1025, 150, 1),   # mixed, K = 1026: P = 4096
    (0, 0.9, 2, 60, 1),       # mixed, K = 3: the shortest transform, P = 16
])
def test_sine_transform_any_size(ft, oracle, kind, gamma, M, N, prec):
    f = wl.random_field((M, N), seed=M + 7 * N)
    ref = oracle.march(kind, 1, gamma, f)
    u = _solve_gpu(ft, kind, gamma, f, precision=prec)
    assert _rel(u, ref) < (1e-12 if prec == 0 else 1e-6)


def test_fp64_four_step_levels(ft, oracle):
    """N = 9000 -> padded 16384: levels s = 4096 use the four-step convolution."""
    M, N = 3, 9000
    f = wl.random_field((M, N), seed=5)
    ref = oracle.march(0, 1, 0.6, f)
    u = _solve_gpu(ft, 0, 0.6, f)
    assert _rel(u, ref) < 1e-12


# With initial data the right-hand side carries scale*u0 (scale = c = tau^-g/Gamma(3-g) for
# the hyperbolic scheme), which cancels against the history down to O(1): two correct
# double evaluations in different summation orders differ by ~eps*scale relative.  The
# cases below keep eps*scale < 3e-13 so that the 1e-12 bound still means "same answer".


def test_space_none_rows_and_initial_data(ft, oracle):
    M, N = 5, 300
    rng = np.random.default_rng(1)
    f = rng.standard_normal((M, N))
    u0 = rng.standard_normal(M)
    phi = rng.standard_normal(M)
    for kind, g in ((0, 0.4), (1, 1.2)):
        ref = oracle.march(kind, 0, g, f, lam=2.5, u0=u0, phi=phi if kind else None)
        u = _solve_gpu(ft, kind, g, f, space=0, lam=2.5, u0=u0, phi=phi if kind else None, tuning=SMALL_TUNE)
        assert _rel(u, ref) < 1e-12


def test_dirichlet_initial_data(ft, oracle):
    M, N = 15, 400
    rng = np.random.default_rng(2)
    f = rng.standard_normal((M, N))
    u0 = rng.standard_normal(M)
    phi = rng.standard_normal(M)
    ref = oracle.march(1, 1, 1.2, f, u0=u0, phi=phi)
    u = _solve_gpu(ft, 1, 1.2, f, u0=u0, phi=phi)
    assert _rel(u, ref) < 1e-12


@pytest.mark.parametrize("kind,gamma,M,N", [(0, 0.7, 31, 3000), (1, 1.5, 63, 2500), (0, 0.2, 15, 5000)])
def test_mixed_precision(ft, oracle, kind, gamma, M, N):
    p = (wl.config_diffusion if kind == 0 else wl.config_wave)(M=M, N=N, gamma=gamma)
    f = wl.materialize(p.source, p.kind, N, M)
    ref = oracle.march(kind, 1, gamma, f)
    u = _solve_gpu(ft, kind, gamma, f, precision=1)
    assert _rel(u, ref) < 1e-6


def test_matvec(ft, oracle):
    import torch
    N = 1000
    rng = np.random.default_rng(4)
    x = rng.standard_normal((5, N))
    with ft.Plan([ft.ProblemSpec(0, 0.7, N, 5, space=0)]) as plan:
        a = plan.weights(0)
        for tr in (False, True):
            y = plan.matvec(0, torch.from_numpy(x).cuda(), transpose=tr)
            plan.sync()
            ref = oracle.toeplitz_matvec(a, x, transpose=tr)
            assert _rel(y.cpu().numpy(), ref) < 1e-12
            yh = plan.matvec(0, x, transpose=tr)  # host buffers
            assert _rel(yh, ref) < 1e-12


def test_weights_vs_oracle(ft, oracle):
    for kind, g, N in ((0, 0.7, 70000), (1, 1.5, 300000), (0, 0.05, 5000), (1, 1.95, 5000)):
        with ft.Plan([ft.ProblemSpec(kind, g, N, 1, space=0)]) as plan:
            a, d = plan.weights(0, with_dgamma=True)
        ref = oracle.toeplitz_column(kind, g, N)
        np.testing.assert_allclose(a, ref, rtol=1e-14, atol=0)
        dref = oracle.toeplitz_column_dgamma(kind, g, N)
        np.testing.assert_allclose(d, dref, rtol=1e-10, atol=1e-12 * np.max(np.abs(dref)))


def test_adjoint_and_gamma_gradient(ft, oracle):
    import torch
    M, N, g = 31, 512, 0.6
    p = wl.config_adjoint(M=M, N=N, gamma=g)
    f = wl.materialize(p.source, p.kind, N, M)
    u_obs = oracle.march(0, 1, 0.55, f)[:, -1] + wl.noise(M, 1e-3, seed=3)
    u = oracle.march(0, 1, g, f)
    dLdu = np.zeros_like(u)
    dLdu[:, -1] = 2 * (u[:, -1] - u_obs)
    lam_ref = oracle.adjoint_march(0, 1, g, dLdu)
    grad_ref = oracle.gamma_gradient(0, g, u, lam_ref)
    with ft.Plan([ft.ProblemSpec(0, g, N, M)]) as plan:
        uu = plan.solve(torch.from_numpy(f).cuda())
        dldf, dg = plan.adjoint(torch.from_numpy(dLdu).cuda(), uu)
    assert _rel(dldf.cpu().numpy(), lam_ref) < 1e-12
    assert abs(dg[0] - grad_ref) <= 1e-9 * abs(grad_ref)


@pytest.mark.parametrize("kind,gamma,M,N,prec", [
    (0, 0.5, 1, 1, 0),      # one step, one point (M+1 = 2: the smallest sine transform, a self pair)
    (1, 1.5, 1, 2, 0),
    (0, 0.7, 3, 5, 1),      # mixed, M+1 = 4
    (1, 1.3, 1, 17, 1),
    (0, 0.6, 7, 16, 0),     # N exactly one minimal block
    (1, 1.7, 2, 1, 0),      # chirp-z transform with a single step
])
def test_degenerate_sizes(ft, oracle, kind, gamma, M, N, prec):
    f = wl.random_field((M, N), seed=17 * M + N)
    ref = oracle.march(kind, 1, gamma, f)
    u = _solve_gpu(ft, kind, gamma, f, precision=prec)
    assert _rel(u, ref) < (1e-12 if prec == 0 else 1e-6)


@pytest.mark.parametrize("kind,gamma,M,N,prec", [
    (0, 0.7, 8191, 40, 1),  # largest power-of-two M+1, mixed
    (1, 1.4, 4095, 40, 0),  # largest power-of-two M+1, double
    (0, 0.6, 4094, 30, 1),  # largest chirp-z M+1 = 4095, mixed
    (1, 1.6, 2046, 30, 0),  # chirp-z M+1 = 2047, double
    (0, 0.45, 4094, 24, 0),  # largest chirp-z M+1 = 4095, double (folded form): P = 8192
    (1, 1.2, 2048, 30, 1),  # mixed chirp-z K = 2049: 2K - 3 = P - 1 at P = 4096
])
def test_largest_sine_transforms(ft, oracle, kind, gamma, M, N, prec):
    f = wl.random_field((M, N), seed=M + N)
    ref = oracle.march(kind, 1, gamma, f)
    u = _solve_gpu(ft, kind, gamma, f, precision=prec)
    assert _rel(u, ref) < (1e-12 if prec == 0 else 1e-6)


@pytest.mark.parametrize("kind,gamma,prec,tol", [(0, 0.6, 0, 1e-13), (1, 1.5, 0, 1e-13),
                                                 (0, 0.6, 1, 1e-9), (1, 1.5, 1, 1e-9)])
def test_longest_line_backward_error(ft, kind, gamma, prec, tol):
    """N = 2^22 (the step limit), two lines without space: the oracle cannot march that far,
    so the check is the backward error of the solve, a property at any size:
    |T u + lambda u - f| <= tol (|a|_1 |u| + lambda |u| + |f|) with T u from the library's
    double circulant-embedded product and a from ftoep_weights."""
    import torch
    N, M, lam = 1 << 22, 2, 1.0
    f = torch.from_numpy(wl.random_field((M, N), seed=kind * 10 + prec)).cuda()
    with ft.Plan([ft.ProblemSpec(kind, gamma, N, M, 0, prec, lam=lam)]) as plan:
        u = plan.solve(f)
        tu = plan.matvec(0, u)
        a = plan.weights(0)
        plan.sync()
    r = tu + lam * u - f
    umax = float(u.abs().max())
    scale = float(np.abs(a).sum()) * umax + lam * umax + float(f.abs().max())
    assert float(r.abs().max()) <= tol * scale
