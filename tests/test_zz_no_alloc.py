"""The allocation-free Toeplitz product (ftoep_matvec_noalloc) against the plan-based
ftoep_matvec, through the C ABI, on consecutive calls.

Callers that cannot allocate device memory (frozen memory budgets, plugins, blocking-
sensitive loops) use ftoep_matvec_noalloc, which keeps its intermediates in a static
device array shared by all calls.  Two calls in a row with different sizes check that
contents left by the previous call never reach a result: the first call (N = 3000) uses
the four-step convolution, the second (N = 1000, transposed) the shared-memory one with
a shorter padding.  This file is collected last on purpose.
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


def test_noalloc_rejects_oversize():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_11593_gb300 import ftoep
    N = 32769
    a = torch.zeros(N, dtype=torch.float64, device="cuda")
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    y = torch.zeros(N, dtype=torch.float64, device="cuda")
    with pytest.raises(ftoep.FtoepError) as ei:
        ftoep.ftoep_matvec_noalloc(a, N, x, y, 1)
    assert ei.value.status == ftoep.FTOEP_EINVAL and "32768" in str(ei.value)
