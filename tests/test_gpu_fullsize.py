"""GPU parity at the full workload sizes, in the launch configuration bench.py times.

The oracle is O(M N^2), so the full fields are checked where the oracle can reach:
* time prefix: the scheme is causal, so the first n0 levels of the full solve equal the
  oracle's full solve of the n0-level problem with the same tau (all spatial points);
* sampled sine modes over the full length: the GPU field is projected onto mode m and
  compared with the oracle's scalar march of that mode;
* modes that the source does not force stay at roundoff level (any size).
"""
import threading

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


def _gpu_solve(ft, p, precision):
    import torch
    f = wl.materialize_torch(p.source, p.kind, p.N, p.M, device="cuda")
    with ft.Plan([ft.ProblemSpec(p.kind, p.gamma, p.N, p.M, p.space, precision)]) as plan:
        u = plan.solve(f)
        plan.sync()
    del f
    return u


def _project_gpu(u, m):
    """Orthonormal sine coefficient of mode m of every time column of the GPU field."""
    import torch
    M = u.shape[0]
    j = torch.arange(1, M + 1, dtype=torch.float64, device=u.device)
    s = torch.sin(torch.remainder(m * j, 2 * (M + 1)) * (np.pi / (M + 1))) * np.sqrt(2.0 / (M + 1))
    return (s @ u).cpu().numpy()


def _oracle_mode(oracle, p, m, chunk=8192):
    """f-hat_m from the source in time chunks, then the scalar march of mode m."""
    fh = np.empty(p.N)
    t_all = wl.time_points(p.kind, p.N, p.T)
    for n0 in range(0, p.N, chunk):
        fc = wl.materialize(p.source, p.kind, p.N, p.M, t=t_all[n0:n0 + chunk])
        fh[n0:n0 + chunk] = oracle.sine_project(fc, m)
    return oracle.march_mode(p.kind, p.gamma, fh, oracle.mode_eigenvalue(m, p.M), T=p.T)


def _oracle_modes_parallel(oracle, p, modes):
    out = {}

    def work(m):
        out[m] = _oracle_mode(oracle, p, m)

    ths = [threading.Thread(target=work, args=(m,)) for m in modes]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    return out


def _oracle_prefix(oracle, p, n0):
    f = wl.materialize(p.source, p.kind, p.N, p.M)[:, :n0] if p.M * p.N <= 2 ** 27 else \
        wl.materialize(p.source, p.kind, p.N, p.M, t=wl.time_points(p.kind, p.N, p.T)[:n0])
    return oracle.march(p.kind, p.space, p.gamma, np.ascontiguousarray(f), T=p.T * n0 / p.N)


def _rel(a, b):
    return float(max(np.linalg.norm(a - b) / np.linalg.norm(b), np.max(np.abs(a - b)) / np.max(np.abs(b))))


def _checked_set_rel(pairs):
    """Relative 2-norm error over a checked set made of several (gpu, reference) parts
    (the time prefix and the full-length sampled modes together)."""
    num = sum(float(np.sum((a - b) ** 2)) for a, b in pairs)
    den = sum(float(np.sum(b ** 2)) for _, b in pairs)
    return (num / den) ** 0.5


# The mixed path's double residual r = f - A u is one Toeplitz product of length 2N over
# the whole line, so its rounding is absolute, at eps times the scale of the whole
# solution.  Early levels, where u is many orders of magnitude smaller than at t = T, are
# therefore accurate relative to max|u| over the field, not relative to their own size.
# Mixed checks use the relative 2-norm over the checked set (prefix + sampled modes) and
# bound the prefix's max error by 1e-6 * max|u| over the field.


def test_config2_diffusion_fp64_full(ft, oracle):
    """gamma = 0.7, M = 1023, N = 65536, double path: <= 1e-12 relative."""
    p = wl.config_diffusion()
    u = _gpu_solve(ft, p, ft.FP64)
    n0 = 4096
    ref = _oracle_prefix(oracle, p, n0)
    assert _rel(u[:, :n0].cpu().numpy(), ref) < 1e-12
    modes = [1, 2, 512, 1023]
    refm = _oracle_modes_parallel(oracle, p, modes)
    umax = float(u.abs().max())
    for m in modes:
        um = _project_gpu(u, m)
        if m == 1:
            assert _rel(um, refm[m]) < 1e-12
        else:
            # unforced modes: the exact discrete answer is 0
            assert np.max(np.abs(um - refm[m])) < 1e-12 * umax
            assert np.max(np.abs(um)) < 1e-13 * umax * 10
    # close to the manufactured solution (O(tau^1.3 + h^2))
    ex = wl.materialize_torch(p.exact, 0, p.N, p.M, device="cuda")
    assert float((u - ex).abs().max()) < 5e-6


def test_config2_diffusion_mixed_full(ft, oracle):
    p = wl.config_diffusion()
    u = _gpu_solve(ft, p, ft.MIXED)
    n0 = 4096
    ref = _oracle_prefix(oracle, p, n0)
    refm = _oracle_modes_parallel(oracle, p, [1, 2])
    up = u[:, :n0].cpu().numpy()
    parts = [(up, ref)] + [(_project_gpu(u, m), refm[m]) for m in (1, 2)]
    assert _checked_set_rel(parts) < 1e-6
    umax = float(u.abs().max())
    assert np.max(np.abs(up - ref)) < 1e-6 * umax


def test_config3_wave_mixed_full(ft, oracle):
    """gamma = 1.5, M = 4095, N = 262144, mixed path: <= 1e-6 relative on the first 4096
    levels (all points) and on the two forced modes over the full length."""
    p = wl.config_wave()
    u = _gpu_solve(ft, p, ft.MIXED)
    n0 = 4096
    ref = _oracle_prefix(oracle, p, n0)
    refm = _oracle_modes_parallel(oracle, p, [1, 3])
    up = u[:, :n0].cpu().numpy()
    parts = [(up, ref)] + [(_project_gpu(u, m), refm[m]) for m in (1, 3)]
    assert _checked_set_rel(parts) < 1e-6
    for m in (1, 3):
        assert _rel(_project_gpu(u, m), refm[m]) < 1e-6
    umax = float(u.abs().max())
    assert np.max(np.abs(up - ref)) < 1e-6 * umax
    for m in (2, 4000):
        assert np.max(np.abs(_project_gpu(u, m))) < 1e-6 * umax


def _all_modes_gpu(u):
    """Every sine mode of the field at once: the orthonormal DST-I matrix (built in double
    from its definition, not by the library) times u, on the GPU -- test-side only."""
    import torch
    M = u.shape[0]
    j = torch.arange(1, M + 1, dtype=torch.int64, device=u.device)
    arg = torch.remainder(j[:, None] * j[None, :], 2 * (M + 1)).to(torch.float64) * (np.pi / (M + 1))
    return (np.sqrt(2.0 / (M + 1)) * torch.sin(arg)) @ u


@pytest.mark.parametrize("prec,forced,tol", [(0, (1,), 1e-12), (1, (1,), 1e-7)])
def test_config2_every_unforced_mode_vanishes(ft, prec, forced, tol):
    """The config-2 source is sin(pi x_j) times a function of time, the m = 1 eigenvector of
    the discrete Laplacian, so the exact discrete solution has no other mode: all 1022 of
    them must stay at the path's rounding level against the forced one."""
    p = wl.config_diffusion()
    u = _gpu_solve(ft, p, prec)
    modal = _all_modes_gpu(u)
    scale = float(modal[0].abs().max())
    keep = [m - 1 for m in forced]
    mask = np.ones(p.M, dtype=bool)
    mask[keep] = False
    import torch
    other = modal[torch.from_numpy(mask).to(modal.device)]
    assert float(other.abs().max()) < tol * scale


def test_config3_every_unforced_mode_vanishes(ft):
    """Config 3 forces modes 1 and 3 only; the other 4093 modes of the mixed solve must stay
    at its rounding level against them."""
    import torch
    p = wl.config_wave()
    u = _gpu_solve(ft, p, ft.MIXED)
    scale = float(u.abs().max())
    worst = 0.0
    for r0 in range(0, p.M, 512):  # row blocks of the projection keep the temporaries small
        M = p.M
        j = torch.arange(1, M + 1, dtype=torch.int64, device=u.device)
        rows = torch.arange(r0 + 1, min(M, r0 + 512) + 1, dtype=torch.int64, device=u.device)
        arg = torch.remainder(rows[:, None] * j[None, :], 2 * (M + 1)).to(torch.float64) * (np.pi / (M + 1))
        S = np.sqrt(2.0 / (M + 1)) * torch.sin(arg)
        modal = S @ u
        for m in (1, 3):
            if r0 < m <= r0 + 512:
                modal[m - 1 - r0] = 0.0
        worst = max(worst, float(modal.abs().max()))
        del modal, S
    assert worst < 1e-7 * scale
