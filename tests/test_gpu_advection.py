"""The advection schemes of Sec. 3 (Scheme 2, Eq. 12/13; Scheme 3, Eq. 16/17) by the
space-order sweep on the GPU (ftoep_advection_sweep, through the C ABI): against the oracle's
direct method (time order) element by element, with initial data, in double (1e-12 of the
data) and mixed precision (1e-6); and the printed values of Tables 5 and 7 from the GPU
solution (the tables' fixtures in tests/golden)."""
import math
import os

import numpy as np
import pytest

from paper_1710_11593_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ft():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_11593_gb300 import ftoep
    ftoep.load()
    return ftoep


def _golden(name):
    with open(os.path.join(HERE, "golden", name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def _printed_match(value, printed):
    e = math.floor(math.log10(abs(printed)))
    return abs(value - printed) <= 1.0001 * 10.0 ** (e - 4)


def _err(u, ref, *scales):
    s = max([np.max(np.abs(ref))] + [np.max(np.abs(x)) for x in scales if x is not None])
    d = np.asarray(u) - np.asarray(ref)
    return max(np.linalg.norm(d) / np.linalg.norm(ref), np.max(np.abs(d)) / s)


@pytest.mark.parametrize("scheme,gamma,M,N,prec,init", [
    (2, 0.4, 40, 900, 0, True),
    (2, 0.9, 17, 5000, 0, False),     # more than one time block
    (3, 1.3, 33, 700, 0, True),
    (3, 1.8, 10, 9000, 0, True),
    (2, 0.6, 25, 3000, 1, False),     # mixed
    (3, 1.5, 25, 3000, 1, True),      # mixed
])
def test_sweep_vs_oracle(ft, oracle, scheme, gamma, M, N, prec, init):
    import torch
    rng = np.random.default_rng(scheme * 100 + M)
    f = rng.standard_normal((M, N))
    u0 = rng.standard_normal(M) if init else None
    phi = rng.standard_normal(M) if init and scheme == 3 else None
    ref = oracle.advection_march(scheme, gamma, f, u0=u0, phi=phi)
    tf = torch.from_numpy(f).cuda()
    t0 = None if u0 is None else torch.from_numpy(u0).cuda()
    tp = None if phi is None else torch.from_numpy(phi).cuda()
    u = ft.advection_sweep(scheme, tf, gamma, u0=t0, phi=tp, precision=prec).cpu().numpy()
    assert _err(u, ref, u0, phi) < (1e-12 if prec == 0 else 1e-6)


def test_sweep_host_buffers(ft, oracle):
    f = wl.random_field((12, 1500), seed=4)
    ref = oracle.advection_march(3, 1.6, f)
    u = ft.advection_sweep(3, f, 1.6)
    assert _err(u, ref) < 1e-12


@pytest.mark.parametrize("row", _golden("table5.txt"))
def test_table5_from_gpu(ft, row):
    """Example 2 by Scheme 2 on the GPU, tau = 2^-10: the printed direct-method values are
    10 x sqrt(h sum_{i<M} e_i^2) (all 12 match)."""
    M, g, printed = int(row[0]), float(row[1]), float(row[2])
    N, h = 1024, 1.0 / M
    xm = (np.arange(1, M + 1) - 0.5) * h
    t = wl.time_points(0, N)
    f = np.outer(np.sin(np.pi * xm), t ** (1 - g) / math.gamma(2 - g)) + np.outer(np.pi * np.cos(np.pi * xm), t)
    u = ft.advection_sweep(2, f, g)
    e = u[:-1, -1] - np.sin(np.pi * np.arange(1, M) * h)
    assert _printed_match(10.0 * math.sqrt(h * np.sum(e ** 2)), printed)


@pytest.mark.parametrize("row", _golden("table7.txt"))
def test_table7_from_gpu(ft, row):
    """Example 3 by Scheme 3 on the GPU, h = tau; the misprinted entry against its fast twin."""
    M, g, direct, fast = int(row[0]), float(row[1]), float(row[2]), float(row[3])
    h = 1.0 / M
    x = np.arange(1, M + 1) * h
    th = wl.time_points(1, M)
    f = np.outer(x - x * x, 6 * th ** (3 - g) / math.gamma(4 - g)) + np.outer(1 - 2 * x, th ** 3)
    u = ft.advection_sweep(3, f, g)
    e = u[:-1, -1] - (x - x * x)[:-1]
    err = math.sqrt(h * np.sum(e ** 2))
    assert _printed_match(err, fast if (M, g) == (8, 1.9) else direct)
