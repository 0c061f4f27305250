"""Runtime around the solve: captured-graph replay of ftoep_solve and the autotuner.

Device-pointer solves: the first call with a pointer set runs directly, the second is
captured (every problem's kernels on the internal streams, fork and join) and launched,
later calls replay the graph.  Checked: direct, captured and replayed results are
bitwise identical; a replay uses the buffers' new contents; a second pointer set gets its
own graph; the launch counter counts the kernels of a replay like those of a direct solve;
instrumentation bypasses the graph.  Plans on the legacy default stream (PyTorch's default)
and batched plans with internal streams are both covered.
"""
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


def _fields(probs):
    import torch
    units = sum(p.M * p.N for p in probs)
    f = torch.empty(units, dtype=torch.float64, device="cuda")
    off = 0
    for p in probs:
        n = p.M * p.N
        wl.materialize_torch(p.source, p.kind, p.N, p.M, device="cuda", out=f[off:off + n].view(p.M, p.N))
        off += n
    return f


def _launches(plan):
    return sum(v[2] for v in plan.profile_read().values())


@pytest.mark.parametrize("nprob,prec", [(1, 0), (1, 1), (6, 1), (6, 0)])
def test_replay_matches_direct(ft, nprob, prec):
    import torch
    probs = wl.config_batched(nprob=nprob, seed=11, n_range=(300, 5000), m_range=(3, 70))
    specs = [ft.ProblemSpec(p.kind, p.gamma, p.N, p.M, p.space, prec) for p in probs]
    f = _fields(probs)
    u = torch.empty_like(f)
    with ft.Plan(specs) as plan:
        outs = []
        for _ in range(4):  # direct, captured, replayed, replayed
            plan.sync()
            u.fill_(float("nan"))
            plan.solve(f, u)
            plan.sync()
            outs.append(u.clone())
        for o in outs[1:]:
            assert torch.equal(o, outs[0])
        # new contents of the same buffers
        f.mul_(-1.5).add_(0.25)
        plan.solve(f, u)
        plan.sync()
        with ft.Plan(specs) as fresh:
            ref = fresh.solve(f)
            fresh.sync()
            fresh.profile(False)
            fresh.solve(f, torch.empty_like(f))
            fresh.sync()
            direct_launches = _launches(fresh)
        assert torch.equal(u, ref)
        # replay counts its kernels
        plan.profile(False)
        plan.solve(f, u)
        plan.sync()
        assert _launches(plan) == direct_launches > 0
        # another output buffer: its own direct run, capture and replay
        u2 = torch.empty_like(f)
        for _ in range(3):
            plan.solve(f, u2)
        plan.sync()
        assert torch.equal(u2, ref)
        # instrumentation bypasses the graph and still gives the same result
        plan.profile(True)
        plan.solve(f, u2)
        plan.sync()
        prof = plan.profile_read()
        plan.profile(False)
        assert torch.equal(u2, ref)
        assert sum(v[1] for v in prof.values()) > 0


def test_replay_on_a_side_stream(ft):
    import torch
    p = wl.config_diffusion(M=31, N=700)
    f = wl.materialize_torch(p.source, p.kind, p.N, p.M, device="cuda")
    s = torch.cuda.Stream()
    spec = ft.ProblemSpec(p.kind, p.gamma, p.N, p.M, p.space, ft.MIXED)
    with torch.cuda.stream(s):
        with ft.Plan([spec], stream=s.cuda_stream) as plan:
            u = torch.empty_like(f)
            res = []
            for _ in range(3):
                plan.solve(f, u)
                res.append(u.clone())
            plan.sync()
    s.synchronize()
    assert torch.equal(res[0], res[1]) and torch.equal(res[1], res[2])


def test_autotune_picks_a_candidate_and_solves(ft, oracle):
    import numpy as np
    probs = wl.config_batched(nprob=5, seed=21, n_range=(500, 9000), m_range=(3, 40))
    specs = [ft.ProblemSpec(p.kind, p.gamma, p.N, p.M, p.space, ft.MIXED) for p in probs]
    tune = ft.ftoep_autotune(specs)
    assert tune["fft_tile"] in (1024, 2048, 4096)
    f = _fields(probs)
    with ft.Plan(specs, tuning=tune) as plan:
        u = plan.solve(f)
        plan.sync()
    off = 0
    for p in probs:
        n = p.M * p.N
        ref = oracle.march(p.kind, p.space, p.gamma, f[off:off + n].view(p.M, p.N).cpu().numpy())
        got = u[off:off + n].view(p.M, p.N).cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-6
        off += n
