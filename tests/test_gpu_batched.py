"""Batched plans: several problems of uneven N, M, gamma and kind in one plan, fields
concatenated in problem order.

Small batch: every problem checked in full against the oracle (double 1e-12, mixed
1e-6 relative).

Full config-4 batch (512 problems), solved in the launch configuration bench.py times,
once in mixed precision and once in double.  Checked problems: the two longest of each
kind, the largest in unknowns, the one with the most interior points (M+1 = 2042, the
chirp-z sine transform), problems 0 and 11, and two drawn at random.  Each is compared
with the oracle on
* its first min(N, 2048) levels, every spatial point (the scheme is causal, so this prefix
  of the full solve is the oracle's full solve of the 2048-level problem with the same tau);
* full-length sine modes: every mode its source forces plus two it does not, each the
  oracle's scalar march of the projected source.
For a problem with N = 2^17 the full-length modes reach every cross-block convolution
level, the running sums of the all-ones part across all 32 time blocks and the correction
sweep over the whole line.  Bars: relative 2-norm over the checked set 1e-6 (mixed) and
1e-12 (double); the max error of the prefix and of every sampled mode within the same
factor of max |u| over the problem's field.
"""
import math
import os
from concurrent.futures import ThreadPoolExecutor

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


def _batch_fields(probs, device="cuda", out=None):
    import torch
    units = sum(p.M * p.N for p in probs)
    f = torch.empty(units, dtype=torch.float64, device=device) if out is None else out
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


def config4_picks(probs, seed=5):
    """Indices of the checked config-4 problems (see the module docstring)."""
    picks = []
    for kind in (0, 1):
        idx = sorted((i for i, p in enumerate(probs) if p.kind == kind), key=lambda i: -probs[i].N)
        picks += idx[:2]
    picks.append(max(range(len(probs)), key=lambda i: probs[i].M * probs[i].N))
    picks.append(max(range(len(probs)), key=lambda i: probs[i].M))
    picks += [0, 11]
    rng = np.random.default_rng(seed)
    picks += [int(i) for i in rng.integers(0, len(probs), 2)]
    return sorted(set(picks))


def _mode_vector(M, m):
    j = np.arange(1, M + 1)
    return np.sqrt(2.0 / (M + 1)) * np.sin(np.remainder(m * j, 2 * (M + 1)) * (math.pi / (M + 1)))


def _projected_source(p, m):
    """f-hat_m over the full length: every term of the source projected onto mode m in
    closed form (sum_j s_m(j) sin(k pi x_j)), times its time factor."""
    s = _mode_vector(p.M, m)
    xs = wl.space_points(p.M)
    tp = wl.time_points(p.kind, p.N)
    fh = np.zeros(p.N)
    for c, pw, k in p.source:
        fh += c * tp ** pw * float(np.dot(s, np.sin(k * math.pi * xs)))
    return fh


def _unforced(p, count=2):
    forced = {k for _, _, k in p.source}
    out = []
    for m in (p.M, p.M // 2, 9, 10, 11, 12):
        if 1 <= m <= p.M and m not in forced and m not in out:
            out.append(m)
        if len(out) == count:
            break
    return out


@pytest.fixture(scope="module")
def config4_reference(oracle):
    """Oracle values of the checked problems: prefix fields and full-length modes, computed
    once (threads: the oracle's C routines release the interpreter lock)."""
    probs = wl.config_batched()
    picks = config4_picks(probs)
    jobs = []
    for i in picks:
        p = probs[i]
        n0 = min(p.N, 2048)
        jobs.append(("prefix", i, n0))
        modes = sorted({k for _, _, k in p.source if k <= p.M}) + _unforced(p)
        for m in modes:
            jobs.append(("mode", i, m))

    def run(job):
        what, i, arg = job
        p = probs[i]
        if what == "prefix":
            fpre = wl.materialize(p.source, p.kind, p.N, p.M, t=wl.time_points(p.kind, p.N)[:arg])
            return job, oracle.march(p.kind, p.space, p.gamma, fpre, T=arg / p.N, nthreads=4)
        fh = _projected_source(p, arg)
        return job, oracle.march_mode(p.kind, p.gamma, fh, oracle.mode_eigenvalue(arg, p.M))

    # longest first
    jobs.sort(key=lambda j: -(probs[j[1]].N ** 2 if j[0] == "mode" else probs[j[1]].M * j[2] ** 2 / 4))
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        res = dict(ex.map(run, jobs))
    return probs, picks, res


@pytest.mark.parametrize("prec,tol,solver", [(1, 1e-6, 0), (0, 1e-12, 0), (1, 1e-6, 3)])
def test_config4_batch_sampled(ft, config4_reference, prec, tol, solver):
    """solver 3: the inverse-series solve for the mixed sub-diffusion problems, the half
    split for the hyperbolic ones."""
    import torch
    probs, picks, res = config4_reference
    f = _batch_fields(probs)
    specs = [ft.ProblemSpec(p.kind, p.gamma, p.N, p.M, p.space, prec) for p in probs]
    with ft.Plan(specs, {"solver": solver} if solver else None) as plan:
        if solver:
            got = [plan.solver(i) for i in picks]
            want = [ft.SOLVER_INVERSE if probs[i].kind == 0 and probs[i].N > 4096 else ft.SOLVER_HALFSPLIT
                    for i in picks]
            assert got == want, (got, want)
        u = plan.solve(f)
        plan.sync()
    del f
    offs = np.cumsum([0] + [p.M * p.N for p in probs])
    for i in picks:
        p = probs[i]
        up = u[offs[i]:offs[i + 1]].view(p.M, p.N)
        n0 = min(p.N, 2048)
        ref = res[("prefix", i, n0)]
        parts = [(up[:, :n0].cpu().numpy(), ref)]
        for (what, j, m), refm in res.items():
            if what == "mode" and j == i:
                s = torch.from_numpy(_mode_vector(p.M, m)).cuda()
                parts.append(((s @ up).cpu().numpy(), refm))
        assert len(parts) >= 5, (i, len(parts))
        num = sum(float(np.sum((a - b) ** 2)) for a, b in parts)
        den = sum(float(np.sum(b ** 2)) for _, b in parts)
        assert (num / den) ** 0.5 < tol, (i, p.kind, p.gamma, p.N, p.M, (num / den) ** 0.5)
        umax = float(up.abs().max())
        assert float(np.max(np.abs(parts[0][0] - ref))) < tol * umax, i
        # every sampled mode on its own, over the full length, against the field's scale
        for (a, b) in parts[1:]:
            assert float(np.max(np.abs(a - b))) < tol * umax, i
    del u
    torch.cuda.empty_cache()
