"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each test ties the oracle to a fact fixed by the paper or by mathematics:
high-precision decimal evaluation of the weight definitions, closed-form
asymptotics and telescoping identities, the values printed in Table 9, convergence
orders against manufactured solutions, a dense linear-algebra solve of the same
scheme built from independently evaluated coefficients, the sine-transform
orthonormality, and the transposition identity behind the adjoint.
"""
import math
import os
from decimal import Decimal, getcontext

import numpy as np
import pytest

from paper_1710_11593_gb300 import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
getcontext().prec = 60


# ----------------------------------------------------------------- decimal references

def d_pow(k, beta):
    if k <= 0:
        return Decimal(0)
    return Decimal(k) ** beta


def d_G(k, g):
    b = Decimal(1) - Decimal(g)
    return d_pow(k + 1, b) - d_pow(k, b)


def d_M(k, g):
    if k < 0:
        return Decimal(0)
    b = Decimal(2) - Decimal(g)
    return d_pow(k + 1, b) - d_pow(k, b)


def d_coef(kind, j, g):
    """Unscaled coefficient of u^{n-j}: Eq. 4/19 (kind 0) and Eq. 17 (kind 1)."""
    if kind == 0:
        return d_G(0, g) if j == 0 else -(d_G(j - 1, g) - d_G(j, g))
    if j == 0:
        return d_M(0, g)
    if j == 1:
        return d_M(1, g) - 2 * d_M(0, g)
    return d_M(j - 2, g) - 2 * d_M(j - 1, g) + d_M(j, g)


def d_scale(kind, g, tau):
    gg = Decimal(g)
    p = (-gg * Decimal(tau).ln()).exp()
    return p / Decimal(repr(math.gamma((2.0 if kind == 0 else 3.0) - g)))


JS = [0, 1, 2, 10, 1000, 65536, 262143]


@pytest.mark.parametrize("g", [0.1, 0.5, 0.7, 0.95])
def test_G_and_l1_coeffs_vs_decimal(oracle, g):
    K = max(JS) + 1
    G = oracle.G(g, K)
    c = oracle.time_coeffs(0, g, K)
    for j in JS:
        ref = float(d_G(j, g))
        assert abs(G[j] - ref) <= 2.3e-16 * abs(ref), (j, G[j], ref)
        refc = float(d_coef(0, j, g))
        assert abs(c[j] - refc) <= 2.3e-16 * abs(refc), (j, c[j], refc)


@pytest.mark.parametrize("g", [1.05, 1.5, 1.9])
def test_M_and_hyperbolic_coeffs_vs_decimal(oracle, g):
    K = max(JS) + 1
    Mv = oracle.Mk(g, K)
    c = oracle.time_coeffs(1, g, K)
    for j in JS:
        ref = float(d_M(j, g))
        assert abs(Mv[j] - ref) <= 2.3e-16 * abs(ref), (j, Mv[j], ref)
        refc = float(d_coef(1, j, g))
        assert abs(c[j] - refc) <= 2.3e-16 * abs(refc), (j, c[j], refc)


@pytest.mark.parametrize("g", [0.1, 0.7, 0.95])
def test_l1_weight_invariants(oracle, g):
    N = 4096
    G = oracle.G(g, N)
    c = oracle.time_coeffs(0, g, N)
    assert G[0] == 1.0
    assert np.all(np.diff(G) < 0), "G_k strictly decreasing (Sec. 3)"
    assert c[0] == 1.0 and np.all(c[1:] < 0), "sign pattern of an M-matrix"
    # telescoping: sum_{j<n} coef_j = G_{n-1}
    cs = np.cumsum(c)
    np.testing.assert_allclose(cs, G, rtol=1e-12, atol=1e-15)
    # large-j asymptotics of the second difference of x^b: b(b-1) j^(b-2) (1 + (b-2)(b-3)/(12 j^2))
    b = 1.0 - g
    for j in (3000, 4000):
        lead = b * (b - 1) * j ** (b - 2) * (1 + (b - 2) * (b - 3) / (12.0 * j * j))
        assert abs(c[j] / lead - 1) < 1e-12


@pytest.mark.parametrize("g", [1.05, 1.5, 1.9])
def test_hyperbolic_weight_invariants(oracle, g):
    N = 4096
    Mv = oracle.Mk(g, N)
    w = oracle.time_coeffs(1, g, N)
    assert Mv[0] == 1.0 and np.all(np.diff(Mv) < 0)
    assert w[0] == 1.0 and w[1] < 0 and np.all(w[2:] > 0)
    # sum_{j<n} w_j = M_{n-1} - M_{n-2} (M_{-1} = 0)
    cs = np.cumsum(w)
    ref = Mv - np.concatenate([[0.0], Mv[:-1]])
    np.testing.assert_allclose(cs, ref, rtol=1e-11, atol=1e-14)
    # third difference centred at j - 1/2: f'''(c) (1 + (b-3)(b-4)/(8 c^2))
    b = 2.0 - g
    for j in (3000, 4000):
        cc = j - 0.5
        lead = b * (b - 1) * (b - 2) * cc ** (b - 3) * (1 + (b - 3) * (b - 4) / (8.0 * cc * cc))
        assert abs(w[j] / lead - 1) < 1e-12


def test_scale_vs_decimal(oracle):
    for kind, g in ((0, 0.7), (0, 0.1), (1, 1.5), (1, 1.9)):
        for N in (8, 1024, 262144):
            ref = float(d_scale(kind, g, 1.0 / N))
            assert abs(oracle.scale(kind, g, 1.0 / N) / ref - 1) < 1e-15


# ----------------------------------------------------------------- Table 9

def _table9_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "table9.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                a, b, c = line.split()
                rows.append((int(a), float(b), float(c)))
    return rows


def _trunc5(x):
    e = math.floor(math.log10(x))
    return math.floor(x / 10 ** (e - 4)) * 10 ** (e - 4)


@pytest.mark.parametrize("h_inv,g,printed", _table9_rows())
def test_table9_direct_method(oracle, h_inv, g, printed):
    """Example 4 / Table 9: final-time discrete L2 error sqrt(h sum_j e_j^N^2)."""
    p = wl.config_table9(h_inv, g)
    f = wl.materialize(p.source, p.kind, p.N, p.M)
    u = oracle.march(p.kind, p.space, g, f)
    ex = wl.materialize(p.exact, p.kind, p.N, p.M)
    h = 1.0 / (p.M + 1)
    err = math.sqrt(h * np.sum((u[:, -1] - ex[:, -1]) ** 2))
    if (h_inv, g) == (256, 0.9):
        # The printed 3.8563e-4 disagrees in the third digit with the direct scheme
        # (3.8503e-4); the table's own rate 1.12 fits both.  Read as a misprint.
        assert abs(err / printed - 1) < 2e-3
    else:
        assert abs(_trunc5(err) - printed) <= 1e-9 * printed, (err, printed)


# ----------------------------------------------------------------- convergence orders

def _rate(e1, e2):
    return math.log2(e1 / e2)


def test_scalar_l1_order(oracle):
    """Config 1 family: D^0.5 u = -u + f, u = t^2; L1 error O(tau^(2-g)) (Lemma 2)."""
    errs = []
    for N in (64, 256, 1024, 4096):
        p = wl.config_scalar(N=N, gamma=0.5)
        f = wl.materialize(p.source, p.kind, N, 1)
        u = oracle.march(p.kind, p.space, 0.5, f, lam=1.0)
        ex = wl.materialize(p.exact, p.kind, N, 1)
        errs.append(np.max(np.abs(u - ex)))
    rates = [_rate(errs[i], errs[i + 1]) / 2 for i in range(len(errs) - 1)]
    assert all(1.4 < r < 1.6 for r in rates), rates
    assert errs[-1] < 2.0 * (1.0 / 4096) ** 1.5


def test_scalar_nonzero_initial_value(oracle):
    """u = 1 + t^2 (u^0 = 1): pins the weight of u^0 in the L1 quotient (G_{n-1})."""
    g = 0.5
    errs = []
    for N in (64, 256, 1024):
        src = wl.manufactured_source([(1.0, 2.0, 0)], g, 0, lam=1.0) + [(1.0, 0.0, 0)]
        f = wl.materialize(src, 0, N, 1)
        u = oracle.march(0, 0, g, f, lam=1.0, u0=np.array([1.0]))
        t = wl.time_points(0, N)
        errs.append(np.max(np.abs(u[0] - (1.0 + t ** 2))))
    rates = [_rate(errs[i], errs[i + 1]) / 2 for i in range(len(errs) - 1)]
    assert all(1.35 < r < 1.65 for r in rates), (errs, rates)


def test_diffusion_order(oracle):
    """Config 2 family (g = 0.7, u = t^2 sin pi x) at h = tau: O(tau^1.3 + h^2)."""
    errs = []
    for n in (16, 32, 64, 128):
        p = wl.config_diffusion(M=n - 1, N=n, gamma=0.7)
        f = wl.materialize(p.source, p.kind, p.N, p.M)
        u = oracle.march(p.kind, p.space, 0.7, f)
        ex = wl.materialize(p.exact, p.kind, p.N, p.M)
        errs.append(math.sqrt(np.sum((u[:, -1] - ex[:, -1]) ** 2) / n))
    rates = [_rate(errs[i], errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(1.2 < r < 2.1 for r in rates), rates


def test_hyperbolic_order(oracle):
    """Config 3 family (g = 1.5, u = t^3 sin pi x + t^3 sin 3 pi x / 9, f at t_{n-1/2},
    spatial term at level n): first-order consistency in time, second in space."""
    errs = []
    for n in (16, 32, 64, 128):
        p = wl.config_wave(M=n - 1, N=n, gamma=1.5)
        f = wl.materialize(p.source, p.kind, p.N, p.M)
        u = oracle.march(p.kind, p.space, 1.5, f)
        ex = wl.materialize(p.exact, 0, p.N, p.M)  # exact values at t_n
        errs.append(math.sqrt(np.sum((u[:, -1] - ex[:, -1]) ** 2) / n))
    rates = [_rate(errs[i], errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(0.8 < r < 2.1 for r in rates), (errs, rates)


def test_hyperbolic_initial_data(oracle):
    """u = 1 + 2t + t^3 (u^0 = 1, u_t(0) = phi = 2): pins the u^0 and phi weights of Eq. 17."""
    g = 1.5
    errs = []
    for N in (64, 256, 1024):
        dc, dp = wl.caputo_power(3.0, g)
        src = [(dc, dp, 0), (1.0, 0.0, 0), (2.0, 1.0, 0), (1.0, 3.0, 0)]  # D^g u + u
        f = wl.materialize(src, 1, N, 1)
        u = oracle.march(1, 0, g, f, lam=1.0, u0=np.array([1.0]), phi=np.array([2.0]))
        t = wl.time_points(0, N)
        errs.append(np.max(np.abs(u[0] - (1.0 + 2 * t + t ** 3))))
    rates = [_rate(errs[i], errs[i + 1]) / 2 for i in range(len(errs) - 1)]
    assert errs[-1] < 1e-2 and all(r > 0.8 for r in rates), (errs, rates)


def _cn_errors(oracle, kind, g, lam, Ns, u0=None, phi=None, space=0, M=1):
    """Max error at the time levels of u = t^3 (+ 1 + 2t with u0 = 1, phi = 2), f at
    t_{n-1/2}.  space 1: the discrete eigenvector sin(pi x_j) with its eigenvalue, so the
    semi-discrete solution is exact and only the time error remains."""
    errs = []
    dc, dp = wl.caputo_power(3.0, g)
    for N in Ns:
        th = wl.time_points(1, N)
        t = wl.time_points(0, N)
        base = (1.0 + 2.0 * th if u0 is not None else 0.0)
        ex = (1.0 + 2.0 * t if u0 is not None else 0.0) + t ** 3
        if space == 0:
            f = (dc * th ** dp + lam * (base + th ** 3))[None, :]
            u = oracle.march(kind, 0, g, f, lam=lam, u0=u0, phi=phi)[0]
            errs.append(np.max(np.abs(u - ex)))
        else:
            x = wl.space_points(M)
            lam1 = oracle.mode_eigenvalue(1, M)
            sx = np.sin(np.pi * x)
            f = np.outer(sx, dc * th ** dp + lam1 * th ** 3)
            u = oracle.march(kind, 1, g, f)
            errs.append(np.max(np.abs(u - np.outer(sx, t ** 3))))
    return errs


@pytest.mark.parametrize("g", [1.5, 1.8])
def test_crank_nicolson_order(oracle, g):
    """Kind 2 (spatial term averaged over levels n and n-1) reaches the O(tau^(3-g)) order
    of the time discretization Eq. 15; kind 1 (spatial term at level n) stays first order.
    u = t^3, scalar (lambda = 5) and the discrete sine eigenvector (M = 15)."""
    Ns = (512, 1024, 2048)
    for space in (0, 1):
        e2 = _cn_errors(oracle, 2, g, 5.0, Ns, space=space, M=15)
        e1 = _cn_errors(oracle, 1, g, 5.0, Ns, space=space, M=15)
        r2, r1 = _rate(e2[-2], e2[-1]), _rate(e1[-2], e1[-1])
        assert abs(r2 - (3.0 - g)) < 0.06, (space, e2, r2)
        assert abs(r1 - 1.0) < 0.1, (space, e1, r1)
        assert e2[-1] < e1[-1] / 2


def test_crank_nicolson_initial_data(oracle):
    """u = 1 + 2t + t^3 (u^0 = 1, phi = 2): the time discretization is exact on 1 + 2t, so
    with correct u^0 and phi terms (including the level-1 average with u^0) the error is
    the error of u = t^3 alone."""
    Ns = (128, 512)
    a = _cn_errors(oracle, 2, 1.5, 5.0, Ns)
    b = _cn_errors(oracle, 2, 1.5, 5.0, Ns, u0=np.array([1.0]), phi=np.array([2.0]))
    np.testing.assert_allclose(b, a, rtol=1e-6)


# ----------------------------------------------------------------- dense brute force

def _dense_system(kind, space, g, M, N, lam=1.0):
    """Kronecker form of the scheme from decimal coefficients: index j*N + n."""
    tau = 1.0 / N
    s = d_scale(kind, g, tau)
    a = [float(s * d_coef(kind, j, g)) for j in range(N)]
    T = np.zeros((N, N))
    for n in range(N):
        for k in range(n + 1):
            T[n, k] = a[n - k]
    if space == 1:
        h = 1.0 / (M + 1)
        K = (np.diag(np.full(M, 2.0)) - np.diag(np.ones(M - 1), 1) - np.diag(np.ones(M - 1), -1)) / h ** 2
    else:
        K = lam * np.eye(M)
    # the spatial operator at level n (kinds 0, 1), or averaged over levels n and n-1
    # (kind 2: half on the diagonal block, half on the block below it)
    Ts = np.eye(N) if kind != 2 else 0.5 * (np.eye(N) + np.eye(N, k=-1))
    A = np.kron(np.eye(M), T) + np.kron(K, Ts)
    if kind == 0:
        wu0 = np.array([float(s * d_G(n - 1, g)) for n in range(1, N + 1)])
        wphi = np.zeros(N)
    else:
        wu0 = np.array([float(s * (d_M(n - 1, g) - d_M(n - 2, g))) for n in range(1, N + 1)])
        wphi = np.array([float(s * Decimal(tau) * d_M(n - 1, g)) for n in range(1, N + 1)])
    return A, wu0, wphi, K


@pytest.mark.parametrize("kind,space,g", [(0, 1, 0.3), (0, 0, 0.8), (1, 1, 1.4), (1, 0, 1.8), (2, 1, 1.6),
                                          (2, 0, 1.2)])
def test_march_vs_dense_solve(oracle, kind, space, g):
    M, N = 6, 20
    rng = np.random.default_rng(7)
    f = rng.standard_normal((M, N))
    u0 = rng.standard_normal(M)
    phi = rng.standard_normal(M) if kind in (1, 2) else None
    A, wu0, wphi, K = _dense_system(kind, space, g, M, N, lam=2.5)
    rhs = f + np.outer(u0, wu0) + (np.outer(phi, wphi) if phi is not None else 0.0)
    if kind == 2:  # the level-1 row averages the spatial operator with u^0
        rhs[:, 0] -= 0.5 * K @ u0
    ref = np.linalg.solve(A, rhs.reshape(-1)).reshape(M, N)
    u = oracle.march(kind, space, g, f, lam=2.5, u0=u0, phi=phi)
    np.testing.assert_allclose(u, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))
    # adjoint: A^T lam = g
    gg = rng.standard_normal((M, N))
    lam_ref = np.linalg.solve(A.T, gg.reshape(-1)).reshape(M, N)
    lam = oracle.adjoint_march(kind, space, g, gg, lam=2.5)
    np.testing.assert_allclose(lam, lam_ref, rtol=0, atol=1e-12 * np.max(np.abs(lam_ref)))


def test_subdiffusion_inverse_nonnegative_and_shift_invariant(oracle):
    """T^-1 >= 0 (M-matrix) and T^-1 e_k = shifted T^-1 e_1 (Toeplitz inverse)."""
    N = 64
    E = np.eye(N)
    U = oracle.march(0, 0, 0.6, E, lam=0.0)  # row k: solution for rhs e_k
    assert np.all(U >= -1e-300)
    for k in range(1, N):
        np.testing.assert_allclose(U[k, k:], U[0, :N - k], rtol=1e-13, atol=0)
        assert np.all(U[k, :k] == 0.0)


def test_causality(oracle):
    rng = np.random.default_rng(3)
    f = rng.standard_normal((5, 40))
    u1 = oracle.march(0, 1, 0.4, f)
    f2 = f.copy()
    f2[:, 25:] = rng.standard_normal((5, 15))
    u2 = oracle.march(0, 1, 0.4, f2)
    assert np.array_equal(u1[:, :25], u2[:, :25])
    # prefix of the full solve = full solve of the prefix problem (same tau)
    u3 = oracle.march(0, 1, 0.4, f[:, :25], T=25.0 / 40.0)
    np.testing.assert_allclose(u3, u1[:, :25], rtol=1e-13, atol=1e-15)


# ----------------------------------------------------------------- sine modes

def test_sine_project_orthonormal(oracle):
    M, N = 31, 5
    j = np.arange(1, M + 1)
    S = np.sqrt(2.0 / (M + 1)) * np.sin(np.pi * np.outer(j, j) / (M + 1))
    np.testing.assert_allclose(S @ S, np.eye(M), atol=1e-14)
    rng = np.random.default_rng(0)
    f = rng.standard_normal((M, N))
    for m in (1, 2, 17, 31):
        np.testing.assert_allclose(oracle.sine_project(f, m), S[m - 1] @ f, atol=1e-13)
    # the sine vector of mode 3 is an eigenvector of the central second difference
    h = 1.0 / (M + 1)
    v = np.sin(3 * np.pi * j * h)
    lap = (2 * v - np.concatenate([[0], v[:-1]]) - np.concatenate([v[1:], [0]])) / h ** 2
    np.testing.assert_allclose(lap, oracle.mode_eigenvalue(3, M) * v, rtol=1e-12)


@pytest.mark.parametrize("kind,g", [(0, 0.7), (1, 1.5), (2, 1.7)])
def test_per_mode_march_matches_full_march(oracle, kind, g):
    M, N = 15, 48
    rng = np.random.default_rng(11)
    f = rng.standard_normal((M, N))
    u = oracle.march(kind, 1, g, f)
    for m in (1, 4, 15):
        fh = oracle.sine_project(f, m)
        uh = oracle.march_mode(kind, g, fh, oracle.mode_eigenvalue(m, M))
        np.testing.assert_allclose(oracle.sine_project(u, m), uh, rtol=0, atol=1e-12 * np.max(np.abs(uh)))


# ----------------------------------------------------------------- adjoint and gradient

@pytest.mark.parametrize("kind,g", [(0, 0.6), (1, 1.3), (2, 1.6)])
def test_adjoint_dot_product(oracle, kind, g):
    M, N = 9, 64
    rng = np.random.default_rng(5)
    f = rng.standard_normal((M, N))
    gg = rng.standard_normal((M, N))
    u = oracle.march(kind, 1, g, f)
    lam = oracle.adjoint_march(kind, 1, g, gg)
    lhs, rhs = np.sum(u * gg), np.sum(f * lam)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.linalg.norm(u) * np.linalg.norm(gg))


def test_gamma_gradient_vs_central_difference(oracle):
    """dL/dg for L = ||u(., T) - u_obs||^2 (config 5 family at M=7, N=64)."""
    M, N, g = 7, 64, 0.6
    p = wl.config_adjoint(M=M, N=N, gamma=g)
    f = wl.materialize(p.source, p.kind, N, M)
    u_obs = oracle.march(0, 1, 0.55, f)[:, -1] + wl.noise(M, 1e-3, seed=2)

    def loss(gam):
        u = oracle.march(0, 1, gam, f)
        return float(np.sum((u[:, -1] - u_obs) ** 2))

    u = oracle.march(0, 1, g, f)
    dLdu = np.zeros_like(u)
    dLdu[:, -1] = 2 * (u[:, -1] - u_obs)
    lam = oracle.adjoint_march(0, 1, g, dLdu)
    grad = oracle.gamma_gradient(0, g, u, lam)
    eps = 1e-6
    fd = (loss(g + eps) - loss(g - eps)) / (2 * eps)
    assert abs(grad - fd) <= 1e-6 * abs(fd), (grad, fd)
    # gradient w.r.t. f: lam (checked on one entry by central differences)
    j, n = 3, 40
    fp, fm = f.copy(), f.copy()
    fp[j, n] += 1e-4
    fm[j, n] -= 1e-4
    lp = float(np.sum((oracle.march(0, 1, g, fp)[:, -1] - u_obs) ** 2))
    lm = float(np.sum((oracle.march(0, 1, g, fm)[:, -1] - u_obs) ** 2))
    assert abs((lp - lm) / 2e-4 - lam[j, n]) <= 1e-6 * abs(lam[j, n])


# ----------------------------------------------------------------- Toeplitz product

def test_toeplitz_matvec_vs_dense(oracle):
    from scipy.linalg import toeplitz
    rng = np.random.default_rng(9)
    N = 77
    a = rng.standard_normal(N)
    x = rng.standard_normal((3, N))
    T = np.tril(toeplitz(a))
    np.testing.assert_allclose(oracle.toeplitz_matvec(a, x), x @ T.T, atol=1e-12)
    np.testing.assert_allclose(oracle.toeplitz_matvec(a, x, transpose=True), x @ T, atol=1e-12)


def _extended_scalar_march(kind, g, N, lam, f):
    """Independent statement of the scalar march in extended precision: weights from mpmath
    at 40 digits (Lemma 1 / Sec. 3 definitions, Eq. 4 and Eq. 17 coefficients), rounded to
    numpy longdouble, levels solved in longdouble."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    gm, tau = mp.mpf(g), mp.mpf(1) / N
    if kind == 0:
        b, sc = 1 - gm, tau ** (-gm) / mp.gamma(2 - gm)
        Gk = lambda k: (k + 1) ** b - (k ** b if k > 0 else 0)
        c = [Gk(0)] + [-(Gk(j - 1) - Gk(j)) for j in range(1, N)]
    else:
        b, sc = 2 - gm, tau ** (-gm) / mp.gamma(3 - gm)
        Mk = lambda k: mp.mpf(0) if k < 0 else (k + 1) ** b - (k ** b if k > 0 else 0)
        c = [Mk(0), Mk(1) - 2 * Mk(0)] + [Mk(j - 2) - 2 * Mk(j - 1) + Mk(j) for j in range(2, N)]
    a = np.array([np.longdouble(mp.nstr(sc * x, 30)) for x in c], dtype=np.longdouble)
    u = np.zeros(N, dtype=np.longdouble)
    for n in range(N):
        hist = np.dot(u[:n], a[n:0:-1]) if n else np.longdouble(0)
        u[n] = (np.longdouble(f[n]) - hist) / (a[0] + np.longdouble(lam))
    return u.astype(np.float64)


@pytest.mark.parametrize("kind,g,lam", [(1, 1.9, 9.55), (1, 1.45, 9.55), (0, 0.7, 9.87)])
def test_march_accuracy_vs_extended_precision(oracle, kind, g, lam):
    """Rounding of the direct march (the paper states no precision): in Eq. 17's form the
    hyperbolic history terms carry tau^-g and cancel to the size of f, and the second-
    difference weights make the discrete solution sensitive to their rounding at about
    eps * N^g.  The oracle (double-double weights and history sums, binary128 level solve)
    must agree with an extended-precision march from 40-digit weights far below the 1e-12
    bar it certifies; plain double history sums miss it by four orders of magnitude here."""
    N = 8192
    t = (np.arange(1, N + 1) - (0.5 if kind == 1 else 0.0)) / N
    f = 1.3 * t ** 1.7 - 0.4 * t ** 2.4
    ref = _extended_scalar_march(kind, g, N, lam, f)
    u = oracle.march(kind, 0, g, f[None, :], lam=lam)[0]
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 2e-13


# ----------------------------------------------------------------- Scheme 1 (Table 1, Theorem 1)

def _table1_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "table1.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                a, b, c = line.split()
                rows.append((int(a), float(b), float(c)))
    return rows


@pytest.mark.parametrize("N,g,printed", _table1_rows())
def test_table1_scheme1(oracle, N, g, printed):
    """Example 1 / Table 1: Scheme 1 (Eq. 7-9) solved densely, L2 error sqrt(tau sum e_i^2)
    against u = t(1-t); the printed values are the errors truncated to 5 digits."""
    t, f, u = wl.two_sided_example1(N, g)
    x = oracle.two_sided_solve(g, f)
    err = math.sqrt(np.sum((x - u) ** 2) / N)
    assert abs(_trunc5(err) - printed) <= 1e-9 * printed, (err, printed)


@pytest.mark.parametrize("g", [0.1, 0.5, 0.9])
def test_scheme1_order(oracle, g):
    """Scheme 1 converges at O(tau^(2-g)) (Sec. 2): the observed rate between N = 2048 and
    4096 is within 0.2 of 2-g (Table 1's last rates: 1.84, 1.50, 1.10)."""
    errs = []
    for N in (2048, 4096):
        t, f, u = wl.two_sided_example1(N, g)
        errs.append(math.sqrt(np.sum((oracle.two_sided_solve(g, f) - u) ** 2) / N))
    assert abs(_rate(errs[0], errs[1]) - (2 - g)) < 0.2


def test_scheme1_matrix_theorem1(oracle):
    """Theorem 1: A is symmetric Toeplitz, and row i's diagonal-dominance margin
    A_ii - sum_{j != i} |A_ij| equals 1 + mu (G_{i-1} + G_{N-1-i}) > 0 (the proof's telescoped
    sums), with G from 60-digit decimal arithmetic."""
    N, g = 40, 0.35
    A = oracle.two_sided_matrix(g, N)
    assert np.array_equal(A, A.T)
    assert all(np.array_equal(np.diag(A, k), np.full(N - 1 - k, A[0, k])) for k in range(N - 1))
    mu = float(d_scale(0, g, 1.0 / N))
    Gd = [float(d_G(k, g)) for k in range(N)]
    for i in range(1, N):
        margin = A[i - 1, i - 1] - (np.sum(np.abs(A[i - 1])) - abs(A[i - 1, i - 1]))
        want = 1 + mu * (Gd[i - 1] + Gd[N - 1 - i])
        assert abs(margin - want) < 1e-12 * (1 + 2 * mu), (i, margin, want)


# ----------------------------------------------------------------- Schemes 2 and 3 (advection)

def _read_golden(name):
    rows = []
    with open(os.path.join(HERE, "golden", name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _printed_match(value, printed):
    """value agrees with a 5-significant-digit printed number (rounded or truncated)."""
    e = math.floor(math.log10(abs(printed)))
    return abs(value - printed) <= 1.0001 * 10.0 ** (e - 4)


def _example2_error(oracle, g, M, N):
    """Scheme 2 on Example 2 (u = t sin pi x, f at (x_{i-1/2}, t_n)): sqrt(h sum_{i<M} e_i^2) at t = 1."""
    h = 1.0 / M
    xm = (np.arange(1, M + 1) - 0.5) * h
    t = wl.time_points(0, N)
    f = np.outer(np.sin(np.pi * xm), t ** (1 - g) / math.gamma(2 - g)) + np.outer(np.pi * np.cos(np.pi * xm), t)
    u = oracle.advection_march(2, g, f)
    e = u[:-1, -1] - np.sin(np.pi * np.arange(1, M) * h)
    return math.sqrt(h * np.sum(e ** 2))


def _example3_error(oracle, g, M, N):
    """Scheme 3 on Example 3 (u = t^3 x (1-x), f at (x_i, t_{n-1/2})): same norm."""
    h = 1.0 / M
    x = np.arange(1, M + 1) * h
    th = wl.time_points(1, N)
    f = np.outer(x - x * x, 6 * th ** (3 - g) / math.gamma(4 - g)) + np.outer(1 - 2 * x, th ** 3)
    u = oracle.advection_march(3, g, f)
    e = u[:-1, -1] - (x - x * x)[:-1]
    return math.sqrt(h * np.sum(e ** 2))


@pytest.mark.parametrize("row", _read_golden("table5.txt"))
def test_table5_scheme2(oracle, row):
    """All 12 direct-method values of Table 5 (the printed values are 10 x the norm)."""
    M, g, printed = int(row[0]), float(row[1]), float(row[2])
    assert _printed_match(10.0 * _example2_error(oracle, g, M, 1024), printed)


@pytest.mark.parametrize("row", _read_golden("table7.txt"))
def test_table7_scheme3(oracle, row):
    """Table 7's direct-method values; the one misprinted entry against its fast-method twin."""
    M, g, direct, fast = int(row[0]), float(row[1]), float(row[2]), float(row[3])
    err = _example3_error(oracle, g, M, M)
    if (M, g) == (8, 1.9):
        assert _printed_match(err, fast) and not _printed_match(err, direct)
    else:
        assert _printed_match(err, direct)


def _dense_advection(scheme, g, M, N):
    """Space-time matrix of scheme 2 or 3 (unknown (i, n) at i*N + n), decimal coefficients."""
    tau = 1.0 / N
    kind = 0 if scheme == 2 else 1
    s = d_scale(kind, g, tau) * (Decimal("0.5") if scheme == 2 else 1)
    a = [float(s * d_coef(kind, j, g)) for j in range(N)]
    T = np.zeros((N, N))
    for n in range(N):
        for k in range(n + 1):
            T[n, k] = a[n - k]
    h = 1.0 / M
    I_M, I_N, S = np.eye(M), np.eye(N), np.eye(M, k=-1)
    A = np.kron(I_M, T) + (np.kron(I_M, I_N) - np.kron(S, I_N)) / h
    if scheme == 2:
        A += np.kron(S, T)
    return A, s


@pytest.mark.parametrize("scheme,g", [(2, 0.3), (2, 0.8), (3, 1.2), (3, 1.8)])
def test_advection_march_vs_dense_solve(oracle, scheme, g):
    M, N = 6, 24
    rng = np.random.default_rng(scheme * 10 + int(10 * g))
    f = rng.standard_normal((M, N))
    u0 = rng.standard_normal(M)
    phi = rng.standard_normal(M) if scheme == 3 else None
    A, s = _dense_advection(scheme, g, M, N)
    rhs = f.copy()
    if scheme == 2:  # c G_{n-1} (u0_i + u0_{i-1}) from both L1 formulas
        wu0 = np.array([float(s * d_G(n - 1, g)) for n in range(1, N + 1)])
        rhs += np.outer(u0 + np.concatenate([[0.0], u0[:-1]]), wu0)
    else:
        tau = Decimal(1) / N
        wu0 = np.array([float(s * (d_M(n - 1, g) - d_M(n - 2, g))) for n in range(1, N + 1)])
        wphi = np.array([float(s * tau * d_M(n - 1, g)) for n in range(1, N + 1)])
        rhs += np.outer(u0, wu0) + np.outer(phi, wphi)
    ref = np.linalg.solve(A, rhs.reshape(-1)).reshape(M, N)
    u = oracle.advection_march(scheme, g, f, u0=u0, phi=phi)
    np.testing.assert_allclose(u, ref, rtol=0, atol=1e-12 * np.max(np.abs(ref)))
