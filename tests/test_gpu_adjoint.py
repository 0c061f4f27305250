"""Differentiation workload: loss = ||u(., T) - u_obs||^2, gradients in f and gamma through
torch.autograd (ftoep_adjoint underneath), against the oracle.

Small case (M = 31, N = 512): oracle adjoint march and oracle gamma-gradient, plus
central differences of the ORACLE forward solve (step 1e-6 in gamma; 1e-4 on f entries
and along one random direction).  Full size (M = 1023, N = 65536): the adjoint is
anti-causal, so its last n0 levels equal the oracle adjoint of the n0-level suffix
problem; sampled modes are marched per mode; the gamma-gradient is the mode-1 term
(u is a pure mode-1 field for this source, the other modes contribute at roundoff).
"""
import math

import numpy as np
import pytest

from paper_1710_11593_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_ft():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_11593_gb300 import autograd, ftoep
    ftoep.load()
    return torch, ftoep, autograd


def _rel(a, b):
    return float(max(np.linalg.norm(a - b) / np.linalg.norm(b), np.max(np.abs(a - b)) / np.max(np.abs(b))))


@pytest.mark.parametrize("recompute", [False, True])
def test_autograd_small_vs_oracle(torch_ft, oracle, recompute):
    torch, ftoep, ag = torch_ft
    M, N, g = 31, 512, 0.6
    p = wl.config_adjoint(M=M, N=N, gamma=g)
    f = wl.materialize(p.source, p.kind, N, M)
    u_obs = oracle.march(0, 1, 0.55, f)[:, -1] + wl.noise(M, 1e-3, seed=8)

    ft_ = torch.from_numpy(f).cuda().requires_grad_(True)
    gt = torch.tensor(g, dtype=torch.float64, requires_grad=True)
    u = ag.fractional_solve(ft_, gt, recompute=recompute)
    loss = torch.sum((u[:, -1] - torch.from_numpy(u_obs).cuda()) ** 2)
    loss.backward()
    dldf = ft_.grad.cpu().numpy()
    dldg = float(gt.grad)

    def oloss(ff, gg):
        uu = oracle.march(0, 1, gg, ff)
        return float(np.sum((uu[:, -1] - u_obs) ** 2))

    uo = oracle.march(0, 1, g, f)
    ug = u.detach().cpu().numpy()
    assert _rel(ug, uo) < 1e-12
    # adjoint field: against the oracle adjoint of the same dL/du.  dL/du = 2(u_T - u_obs)
    # is a small difference of nearly equal fields, so it carries the forward rounding
    # amplified by |u|/|u - u_obs|; comparing with the adjoint of the oracle's dL/du would
    # test that amplification instead of the adjoint solve.
    dLdu_g = np.zeros_like(uo)
    dLdu_g[:, -1] = 2 * (ug[:, -1] - u_obs)
    assert _rel(dldf, oracle.adjoint_march(0, 1, g, dLdu_g)) < 1e-12
    dLdu = np.zeros_like(uo)
    dLdu[:, -1] = 2 * (uo[:, -1] - u_obs)
    lam = oracle.adjoint_march(0, 1, g, dLdu)
    assert _rel(dldf, lam) < 1e-9
    grad_ref = oracle.gamma_gradient(0, g, uo, lam)
    assert abs(dldg - grad_ref) <= 1e-9 * abs(grad_ref)
    # central differences of the oracle forward
    fd = (oloss(f, g + 1e-6) - oloss(f, g - 1e-6)) / 2e-6
    assert abs(dldg - fd) <= 1e-6 * abs(fd)
    rng = np.random.default_rng(4)
    for _ in range(8):
        j, n = int(rng.integers(M)), int(rng.integers(N))
        fp, fm = f.copy(), f.copy()
        fp[j, n] += 1e-4
        fm[j, n] -= 1e-4
        fdj = (oloss(fp, g) - oloss(fm, g)) / 2e-4
        assert abs(fdj - dldf[j, n]) <= 1e-6 * max(abs(fdj), 1e-3 * np.max(np.abs(dldf)))
    d = rng.standard_normal(f.shape)
    fdd = (oloss(f + 1e-5 * d, g) - oloss(f - 1e-5 * d, g)) / 2e-5
    assert abs(fdd - float(np.sum(d * dldf))) <= 1e-6 * abs(fdd)


def test_adjoint_hyperbolic_small(torch_ft, oracle):
    torch, ftoep, ag = torch_ft
    M, N, g = 15, 400, 1.4
    rng = np.random.default_rng(12)
    f = rng.standard_normal((M, N))
    gg = rng.standard_normal((M, N))
    with ftoep.Plan([ftoep.ProblemSpec(1, g, N, M)]) as plan:
        u = plan.solve(torch.from_numpy(f).cuda())
        dldf, dg = plan.adjoint(torch.from_numpy(gg).cuda(), u)
    uo = oracle.march(1, 1, g, f)
    lam = oracle.adjoint_march(1, 1, g, gg)
    assert _rel(dldf.cpu().numpy(), lam) < 1e-11
    ref = oracle.gamma_gradient(1, g, uo, lam)
    assert abs(dg[0] - ref) <= 1e-8 * abs(ref)


def test_config5_adjoint_full(torch_ft, oracle):
    """gamma = 0.6, M = 1023, N = 65536; u_obs from the oracle's mode-1 march at 0.55 plus
    N(0, 1e-3^2) noise."""
    torch, ftoep, ag = torch_ft
    p = wl.config_adjoint()
    M, N, g = p.M, p.N, p.gamma
    x = wl.space_points(M)
    s1 = np.sqrt(2.0 / (M + 1)) * np.sin(math.pi * np.arange(1, M + 1) / (M + 1))
    # the source is sin(pi x) times a time profile: mode 1 only
    tpts = wl.time_points(0, N)
    prof = sum(c * tpts ** pw for c, pw, k in p.source)
    fhat1 = prof * float(np.dot(s1, np.sin(math.pi * x)))
    lam1 = oracle.mode_eigenvalue(1, M)
    uh55 = oracle.march_mode(0, 0.55, fhat1, lam1)
    u_obs = uh55[-1] * s1 + wl.noise(M, 1e-3, seed=21)
    uh = oracle.march_mode(0, g, fhat1, lam1)

    f = wl.materialize_torch(p.source, p.kind, N, M, device="cuda")
    # oracle adjoint input: dL/du = 2 (u(T) - u_obs) at the last level, from the oracle's u.
    # (Built from the GPU's own u instead, it would differ by the forward rounding
    # amplified by |u| / |u(T) - u_obs| ~ 20, which is not an error of the adjoint.)
    gT = 2.0 * (uh[-1] * s1 - u_obs)
    G = torch.zeros_like(f)
    G[:, -1] = torch.from_numpy(gT).cuda()
    with ftoep.Plan([ftoep.ProblemSpec(0, g, N, M)]) as plan:
        dldf, _ = plan.adjoint(G, None, want_gamma=False)
        plan.sync()
    # suffix: last n0 levels, all points (the adjoint is anti-causal)
    n0 = 2048
    gs = np.zeros((M, n0))
    gs[:, -1] = gT
    lam_suffix = oracle.adjoint_march(0, 1, g, gs, T=n0 / N)
    assert _rel(dldf[:, N - n0:].cpu().numpy(), lam_suffix) < 1e-12
    # sampled modes over the full length
    jj = torch.arange(1, M + 1, dtype=torch.float64, device="cuda")
    for m in (1, 2, 700):
        sm = np.sqrt(2.0 / (M + 1)) * np.sin(math.pi * m * np.arange(1, M + 1) / (M + 1))
        ghat = np.zeros(N)
        ghat[-1] = float(np.dot(sm, gT))
        lam_m = oracle.adjoint_march(0, 0, g, ghat[None, :], lam=oracle.mode_eigenvalue(m, M))[0]
        smt = torch.sin(torch.remainder(m * jj, 2 * (M + 1)) * (math.pi / (M + 1))) * math.sqrt(2.0 / (M + 1))
        got = (smt @ dldf).cpu().numpy()
        if m == 1:
            lam_1 = lam_m
            assert _rel(got, lam_m) < 1e-12
        else:
            # noise-driven modes, measured on the scale of the field (mode 1)
            assert np.max(np.abs(got - lam_m)) < 1e-12 * np.max(np.abs(lam_1))
    # gradients through torch.autograd (dL/du from the GPU forward)
    gt = torch.tensor(g, dtype=torch.float64, requires_grad=True)
    fr = f.clone().requires_grad_(True)
    u = ag.fractional_solve(fr, gt)
    loss = torch.sum((u[:, -1] - torch.from_numpy(u_obs).cuda()) ** 2)
    loss.backward()
    # gamma-gradient: mode-1 term
    grad_ref = oracle.gamma_gradient(0, g, uh[None, :], lam_1[None, :])
    assert abs(float(gt.grad) - grad_ref) <= 1e-9 * abs(grad_ref)


def test_autograd_backward_twice_and_plan_reuse(torch_ft):
    """retain_graph: a second backward pass through the same graph gives the same gradients
    (the graph keeps its plan); a second forward pass of the same problem reuses the plan."""
    torch, ftoep, ag = torch_ft
    M, N, g = 15, 300, 0.4
    f = torch.from_numpy(wl.random_field((M, N), seed=21)).cuda().requires_grad_(True)
    gt = torch.tensor(g, dtype=torch.float64, requires_grad=True)
    ag.clear_plan_cache()
    u = ag.fractional_solve(f, gt)
    loss = torch.sum(u[:, -1] ** 2)
    loss.backward(retain_graph=True)
    g1f, g1g = f.grad.clone(), gt.grad.clone()
    f.grad = None
    gt.grad = None
    loss.backward()
    assert torch.equal(f.grad, g1f) and torch.equal(gt.grad, g1g)
    u2 = ag.fractional_solve(f, gt)
    assert u2.grad_fn is not None and torch.equal(u2, u)
    assert len(ag._plans) == 1
    ag.clear_plan_cache()


@pytest.mark.parametrize("kind,gamma", [(0, 0.45), (1, 1.5)])
def test_adjoint_of_mixed_plan_runs_in_double(torch_ft, oracle, kind, gamma):
    """A mixed-precision plan's adjoint solves in double (its own double block-inverse
    spectra): the oracle's transposed march at 1e-12, several time blocks."""
    torch, ftoep, _ = torch_ft
    M, N = 31, 3000
    rng = np.random.default_rng(21 + kind)
    f = rng.standard_normal((M, N))
    gg = rng.standard_normal((M, N))
    with ftoep.Plan([ftoep.ProblemSpec(kind, gamma, N, M, 1, ftoep.MIXED)], {"fft_tile": 512}) as plan:
        u = plan.solve(torch.from_numpy(f).cuda())
        dldf, dg = plan.adjoint(torch.from_numpy(gg).cuda(), u)
        plan.sync()
        u, dldf = u.cpu().numpy(), dldf.cpu().numpy()
    lam = oracle.adjoint_march(kind, 1, gamma, gg)
    assert _rel(dldf, lam) < 1e-12
    ref = oracle.gamma_gradient(kind, gamma, oracle.march(kind, 1, gamma, f), lam)
    assert abs(dg[0] - ref) <= 1e-8 * abs(ref)
