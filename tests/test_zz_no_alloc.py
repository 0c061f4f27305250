"""The allocation-free Toeplitz product (ftoep_matvec_noalloc) against the plan-based
ftoep_matvec, through the C ABI, on consecutive calls.

Callers that cannot allocate device memory (frozen memory budgets, plugins, blocking-
sensitive loops) use ftoep_matvec_noalloc, which keeps its intermediates in a static
device array shared by all calls.  Two calls in a row with different sizes check that
contents left by the previous call never reach a result: the first call (N = 3000) uses
the four-step convolution, the second (N = 1000, transposed) the shared-memory one with
a shorter padding.  The longest supported line (N = 32768: a circulant of 65536, the
largest twiddle table, every region of the static array at full extent) runs with 17
lines (two batches of the array's 16 lines, the last one a single line), against the plan
product and against the oracle's dense product on sampled lines.  This file is collected
last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rel(u, ref):
    return float(np.linalg.norm(u - ref) / np.linalg.norm(ref))


def test_noalloc_matvec_matches_plan_matvec():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_11593_gb300 import ftoep
    ftoep.load()
    rng = np.random.default_rng(17)
    cases = [(3000, 21, False, 0.7), (1000, 5, True, 0.3), (5000, 3, False, 0.5)]
    for N, nlines, transpose, g in cases:
        with ftoep.Plan([ftoep.ProblemSpec(0, g, N, nlines, space=ftoep.SPACE_NONE)]) as plan:
            a = plan.weights(0)
            x = torch.from_numpy(rng.standard_normal((nlines, N))).cuda()
            y_ref = plan.matvec(0, x, transpose=transpose)
            plan.sync()
        a_d = torch.from_numpy(a).cuda()
        y = torch.full_like(x, float("nan"))
        ftoep.ftoep_matvec_noalloc(a_d, N, x, y, nlines, transpose)
        torch.cuda.synchronize()
        assert _rel(y.cpu().numpy(), y_ref.cpu().numpy()) < 1e-12, (N, nlines, transpose)


def test_noalloc_longest_line_against_oracle(oracle):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_11593_gb300 import ftoep
    ftoep.load()
    N, nlines, g = 32768, 17, 0.6
    rng = np.random.default_rng(23)
    xh = rng.standard_normal((nlines, N))
    for transpose in (True, False):
        with ftoep.Plan([ftoep.ProblemSpec(0, g, N, nlines, space=ftoep.SPACE_NONE)]) as plan:
            a = plan.weights(0)
            x = torch.from_numpy(xh).cuda()
            y_ref = plan.matvec(0, x, transpose=transpose).cpu().numpy()
            plan.sync()
        a_d = torch.from_numpy(a).cuda()
        y = torch.full_like(x, float("nan"))
        for _ in range(2):  # two calls in a row on the same array
            ftoep.ftoep_matvec_noalloc(a_d, N, x, y, nlines, transpose)
        torch.cuda.synchronize()
        yn = y.cpu().numpy()
        assert _rel(yn, y_ref) < 1e-12, transpose
        for line in (0, 8, 16):
            ref = oracle.toeplitz_matvec(a, xh[line], transpose=transpose)
            assert _rel(yn[line], ref) < 1e-12, (transpose, line)


def test_noalloc_refuses_host_buffers():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_11593_gb300 import ftoep
    N = 256
    a = torch.ones(N, dtype=torch.float64, device="cuda")
    x_host = torch.ones(N, dtype=torch.float64)
    y = torch.zeros(N, dtype=torch.float64, device="cuda")
    with pytest.raises(ftoep.FtoepError) as ei:
        ftoep.ftoep_matvec_noalloc(a, N, x_host, y, 1)
    assert ei.value.status == ftoep.FTOEP_EINVAL and "device" in str(ei.value)
    torch.cuda.synchronize()
    assert float(y.abs().max()) == 0.0


def test_noalloc_rejects_oversize():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_11593_gb300 import ftoep
    N = 32768
    ok = torch.zeros(N, dtype=torch.float64, device="cuda")
    ftoep.ftoep_matvec_noalloc(ok, N, ok.clone(), torch.empty_like(ok), 1)
    torch.cuda.synchronize()
    N = 32769
    a = torch.zeros(N, dtype=torch.float64, device="cuda")
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    y = torch.zeros(N, dtype=torch.float64, device="cuda")
    with pytest.raises(ftoep.FtoepError) as ei:
        ftoep.ftoep_matvec_noalloc(a, N, x, y, 1)
    assert ei.value.status == ftoep.FTOEP_EINVAL and "32768" in str(ei.value)
