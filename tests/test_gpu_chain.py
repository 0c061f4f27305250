"""The persistent per-pair solve (scheduler FTOEP_SCHED_CHAIN) against the per-level
launches and against the oracle.

The chain runs the same block solves and cross-block convolutions as the per-level
launches (same bodies, same FFT splits, same order per pair), only one pair per block
through the whole recursion, so the two agree to rounding (the bodies compile separately,
so the last bits may differ).  Sizes reach the four-step levels inside the chain (2s above
the shared-memory length: N = 40000 has levels up to 2s = 65536), the chirp-z sine
transform (M+1 not a power of two), both kinds and both precisions; batches check every
problem against the oracle, also with host buffers (through the plan's device copies of the
fields, and staged one problem at a time around the chain launches), with initial data, and
split into several groups by a small memory budget.
"""
import os

import numpy as np
import pytest

from paper_1710_11593_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ft():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_11593_gb300 import ftoep
    ftoep.load()
    return ftoep


def _rel(a, b):
    return float(max(np.linalg.norm(a - b) / np.linalg.norm(b), np.max(np.abs(a - b)) / np.max(np.abs(b))))


def _check(a, b, tol, what):
    """Relative 2-norm error (the error measure of the configs) below tol, the max error
    relative to max |b| below 3 tol (it weighs the smallest levels of a line fully)."""
    r2 = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    rm = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
    assert r2 < tol and rm < 3 * tol, (what, r2, rm)


def _solve(ft, specs, f, sched, **kw):
    # the half-split solver: the chain runs every pair's block solves and levels
    with ft.Plan(specs, tuning={"scheduler": sched, "solver": ft.SOLVER_HALFSPLIT}) as plan:
        u = plan.solve(f, **kw)
        plan.sync()
    return u


@pytest.mark.parametrize("kind,gamma,M,N,prec", [
    (0, 0.7, 31, 40000, 0), (1, 1.5, 30, 40000, 1), (0, 0.35, 100, 9000, 1), (1, 1.2, 63, 17000, 0),
    (0, 0.5, 1, 70000, 1),
])
def test_chain_matches_levels(ft, kind, gamma, M, N, prec):
    import torch
    f = torch.from_numpy(wl.random_field((M, N), seed=M + N)).cuda()
    spec = ft.ProblemSpec(kind, gamma, N, M, 1, prec)
    ul = _solve(ft, [spec], f, ft.SCHED_LEVELS)
    uc = _solve(ft, [spec], f, ft.SCHED_CHAIN)
    d = float((uc - ul).abs().max() / ul.abs().max())
    assert d < (1e-13 if prec == 0 else 1e-12), d


def _batch(probs):
    units = sum(p.M * p.N for p in probs)
    f = np.empty(units)
    off = 0
    for p in probs:
        n = p.M * p.N
        f[off:off + n] = wl.materialize(p.source, p.kind, p.N, p.M).ravel()
        off += n
    return f


@pytest.mark.parametrize("prec,tol,host", [(0, 1e-12, False), (1, 1e-6, False), (0, 1e-12, True), (1, 1e-6, True),
                                           (0, 1e-12, "staged"), (1, 1e-6, "staged")])
def test_chain_batch_vs_oracle(ft, oracle, monkeypatch, prec, tol, host):
    """Device buffers; host buffers with the plan's device copies of the fields (f in once,
    u out once); host buffers through the staging arrays (FTOEP_HOST_STAGED)."""
    import torch
    if host == "staged":
        monkeypatch.setenv("FTOEP_HOST_STAGED", "1")
    probs = wl.config_batched(nprob=9, seed=31, n_range=(300, 12000), m_range=(3, 40))
    fh = _batch(probs)
    specs = [ft.ProblemSpec(p.kind, p.gamma, p.N, p.M, p.space, prec) for p in probs]
    f = fh if host else torch.from_numpy(fh).cuda()
    u = _solve(ft, specs, f, ft.SCHED_CHAIN)
    uh = u if host else u.cpu().numpy()
    off = 0
    for p in probs:
        n = p.M * p.N
        ref = oracle.march(p.kind, p.space, p.gamma, fh[off:off + n].reshape(p.M, p.N))
        _check(uh[off:off + n].reshape(p.M, p.N), ref, tol, (p.kind, p.gamma, p.N, p.M))
        off += n


def test_chain_groups(ft, oracle, monkeypatch):
    """A budget of one problem's pair arrays puts every problem in its own group."""
    import torch
    probs = wl.config_batched(nprob=5, seed=41, n_range=(500, 6000), m_range=(7, 30))
    fh = _batch(probs)
    monkeypatch.setenv("FTOEP_CHAIN_BUDGET", "1")
    for prec, tol in ((0, 1e-12), (1, 1e-6)):
        specs = [ft.ProblemSpec(p.kind, p.gamma, p.N, p.M, p.space, prec) for p in probs]
        u = _solve(ft, specs, torch.from_numpy(fh).cuda(), ft.SCHED_CHAIN).cpu().numpy()
        off = 0
        for p in probs:
            n = p.M * p.N
            ref = oracle.march(p.kind, p.space, p.gamma, fh[off:off + n].reshape(p.M, p.N))
            _check(u[off:off + n].reshape(p.M, p.N), ref, tol, (prec, p.kind, p.N, p.M))
            off += n


# With initial data the difference form solves for v = d_t u with right-hand side
# f - S u0 (S u0 up to 4/h^2 |u0|), and u = u0 + tau cumsum(v) cancels u0 against the sum:
# when the solution decays far below u0 its rounding is eps times the data's scale, not
# eps times |u|.  The double bar is therefore taken against the scale of the data,
# max(max |u|, max |u0|, T max |phi|).
def test_chain_initial_data(ft, oracle, monkeypatch):
    """u0 and phi enter the right-hand side and the mixed residual; two groups."""
    import torch
    probs = wl.config_batched(nprob=4, seed=43, n_range=(200, 400), m_range=(7, 30), g_sub=(0.3, 0.6),
                              g_hyp=(1.1, 1.25))
    fh = _batch(probs)
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal(sum(p.M for p in probs))
    phi = rng.standard_normal(sum(p.M for p in probs))
    monkeypatch.setenv("FTOEP_CHAIN_BUDGET", str(1 << 16))
    for prec, tol in ((0, 1e-12), (1, 1e-6)):
        specs = [ft.ProblemSpec(p.kind, p.gamma, p.N, p.M, p.space, prec) for p in probs]
        u = _solve(ft, specs, torch.from_numpy(fh).cuda(), ft.SCHED_CHAIN, u0=torch.from_numpy(u0).cuda(),
                   phi=torch.from_numpy(phi).cuda()).cpu().numpy()
        off = voff = 0
        for p in probs:
            n = p.M * p.N
            ref = oracle.march(p.kind, p.space, p.gamma, fh[off:off + n].reshape(p.M, p.N), u0=u0[voff:voff + p.M],
                               phi=phi[voff:voff + p.M] if p.kind == 1 else None)
            got = u[off:off + n].reshape(p.M, p.N)
            scale = max(np.max(np.abs(ref)), np.max(np.abs(u0[voff:voff + p.M])),
                        np.max(np.abs(phi[voff:voff + p.M])) if p.kind == 1 else 0.0)
            assert np.max(np.abs(got - ref)) < tol * scale, (prec, p.kind, p.N, p.M)
            if prec == 1:
                _check(got, ref, tol, (prec, p.kind, p.N, p.M))
            off += n
            voff += p.M


def test_forced_allocation_failure_reports_enomem(ft, monkeypatch):
    """Host-side fault injection: the plan's allocations fail after the first few; creation
    returns FTOEP_ENOMEM, frees what it took, and the next plan works."""
    import torch
    spec = ft.ProblemSpec(0, 0.5, 2000, 15, 1, 0)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in (0, 3, 12):
        monkeypatch.setenv("FTOEP_FAIL_ALLOC_AFTER", str(k))
        with pytest.raises(ft.FtoepError) as ei:
            ft.Plan([spec])
        assert ei.value.status == ft.FTOEP_ENOMEM and "FTOEP_FAIL_ALLOC_AFTER" in str(ei.value)
    monkeypatch.delenv("FTOEP_FAIL_ALLOC_AFTER")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)
    f = torch.ones(15 * 2000, dtype=torch.float64, device="cuda")
    with ft.Plan([spec]) as plan:
        plan.solve(f)
        plan.sync()
