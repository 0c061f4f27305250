"""Batched plans: several problems of uneven N, M, gamma and kind in one plan (run on the
plan's internal streams), fields concatenated in problem order.

Small batch: every problem checked in full against the oracle (double 1e-12, mixed
1e-6 relative).  Full config-4 batch (512 problems, mixed): sampled problems checked on
their first min(N, 1024) levels (all points; causality) and on one forced mode over the
full length, with the relative 2-norm over the checked set <= 1e-6.
"""
import math

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


def _batch_fields(probs, device="cuda"):
    import torch
    units = sum(p.M * p.N for p in probs)
    f = torch.empty(units, dtype=torch.float64, device=device)
    off = 0
    for p in probs:
        n = p.M * p.N
        wl.materialize_torch(p.source, p.kind, p.N, p.M, device=device, out=f[off:off + n].view(p.M, p.N))
        off += n
    return f


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6)])
def test_small_batch_every_problem(ft, oracle, prec, tol):
    probs = wl.config_batched(nprob=10, seed=99, n_range=(64, 1500), m_range=(3, 70))
    f = _batch_fields(probs)
    specs = [ft.ProblemSpec(p.kind, p.gamma, p.N, p.M, p.space, prec) for p in probs]
    with ft.Plan(specs) as plan:
        u = plan.solve(f)
        plan.sync()
    off = 0
    for p in probs:
        n = p.M * p.N
        fp = f[off:off + n].view(p.M, p.N).cpu().numpy()
        up = u[off:off + n].view(p.M, p.N).cpu().numpy()
        ref = oracle.march(p.kind, p.space, p.gamma, fp)
        assert _rel(up, ref) < tol, (p.kind, p.gamma, p.N, p.M)
        off += n


def test_config4_batch_sampled(ft, oracle):
    import torch
    probs = wl.config_batched()
    f = _batch_fields(probs)
    specs = [ft.ProblemSpec(p.kind, p.gamma, p.N, p.M, p.space, ft.MIXED) for p in probs]
    with ft.Plan(specs) as plan:
        u = plan.solve(f)
        plan.sync()
    offs = np.cumsum([0] + [p.M * p.N for p in probs])
    rng = np.random.default_rng(5)
    picks = sorted(set([0, 511] + [int(i) for i in rng.integers(0, 512, 4)]))
    for i in picks:
        p = probs[i]
        up = u[offs[i]:offs[i + 1]].view(p.M, p.N)
        n0 = min(p.N, 1024)
        fpre = wl.materialize(p.source, p.kind, p.N, p.M, t=wl.time_points(p.kind, p.N)[:n0])
        ref = oracle.march(p.kind, p.space, p.gamma, fpre, T=n0 / p.N)
        parts = [(up[:, :n0].cpu().numpy(), ref)]
        if p.N <= 20000:
            m = p.source[0][2]
            s = np.sqrt(2.0 / (p.M + 1)) * np.sin(math.pi * m * np.arange(1, p.M + 1) / (p.M + 1))
            fh = np.zeros(p.N)
            tp = wl.time_points(p.kind, p.N)
            xs = wl.space_points(p.M)
            for c, pw, k in p.source:
                fh += c * tp ** pw * float(np.dot(s, np.sin(k * math.pi * xs)))
            refm = oracle.march_mode(p.kind, p.gamma, fh, oracle.mode_eigenvalue(m, p.M))
            st = torch.from_numpy(s).cuda()
            parts.append(((st @ up).cpu().numpy(), refm))
        num = sum(float(np.sum((a - b) ** 2)) for a, b in parts)
        den = sum(float(np.sum(b ** 2)) for _, b in parts)
        assert (num / den) ** 0.5 < 1e-6, (i, p.kind, p.gamma, p.N, p.M)
        umax = float(up.abs().max())
        assert float(np.max(np.abs(parts[0][0] - ref))) < 1e-6 * umax
