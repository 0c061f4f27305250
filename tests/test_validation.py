"""Argument checks of the C ABI (host logic, no GPU needed): every invalid problem or
tuning is rejected by ftoep_create / ftoep_autotune with FTOEP_EINVAL, sizes beyond the
sine-transform and step limits with FTOEP_EUNSUPPORTED, before any device work."""
import pytest

from paper_1710_11593_gb300 import ftoep


def _spec(**kw):
    d = dict(kind=0, gamma=0.5, N=64, M=7, space=1, precision=0)
    d.update(kw)
    return ftoep.ProblemSpec(d["kind"], d["gamma"], d["N"], d["M"], d["space"], d["precision"],
                             **{k: v for k, v in d.items() if k in ("T", "L", "lam")})


@pytest.mark.parametrize("kw,status,msg", [
    (dict(kind=0, gamma=1.0), ftoep.FTOEP_EINVAL, "not in (0,1)"),
    (dict(kind=0, gamma=0.0), ftoep.FTOEP_EINVAL, "not in (0,1)"),
    (dict(kind=1, gamma=0.5), ftoep.FTOEP_EINVAL, "not in (1,2)"),
    (dict(kind=1, gamma=2.0), ftoep.FTOEP_EINVAL, "not in (1,2)"),
    (dict(kind=2, gamma=0.5), ftoep.FTOEP_EINVAL, "not in (1,2)"),
    (dict(kind=2, gamma=2.0), ftoep.FTOEP_EINVAL, "not in (1,2)"),
    (dict(kind=3, gamma=1.5), ftoep.FTOEP_EINVAL, "unknown kind"),
    (dict(space=2), ftoep.FTOEP_EINVAL, "unknown space"),
    (dict(precision=3), ftoep.FTOEP_EINVAL, "unknown precision"),
    (dict(N=0), ftoep.FTOEP_EINVAL, "must be >= 1"),
    (dict(M=0), ftoep.FTOEP_EINVAL, "must be >= 1"),
    (dict(T=0.0), ftoep.FTOEP_EINVAL, "T must be > 0"),
    (dict(T=float("nan")), ftoep.FTOEP_EINVAL, "T must be > 0"),
    (dict(L=-1.0), ftoep.FTOEP_EINVAL, "L must be > 0"),
    (dict(space=0, lam=-1.0), ftoep.FTOEP_EINVAL, "lambda must be >= 0"),
    (dict(N=(1 << 22) + 1), ftoep.FTOEP_EUNSUPPORTED, "N > 2^22"),
    (dict(M=8192, precision=1), ftoep.FTOEP_EUNSUPPORTED, "M+1 = 8193"),   # above the power-of-two mixed limit
    (dict(M=4096, precision=0), ftoep.FTOEP_EUNSUPPORTED, "M+1 = 4097"),   # chirp-z double limit 4096
    (dict(M=4200, precision=1), ftoep.FTOEP_EUNSUPPORTED, "M+1 = 4201"),   # chirp-z mixed limit 4096
])
def test_invalid_problem_rejected(kw, status, msg):
    with pytest.raises(ftoep.FtoepError) as ei:
        ftoep.ftoep_create([_spec(**kw)], None, 0)
    assert ei.value.status == status
    assert msg in str(ei.value)


@pytest.mark.parametrize("tune,msg", [
    ({"leaf": 3}, "leaf"),
    ({"leaf": 32}, "leaf"),
    ({"fft_tile": 8}, "fft_tile"),
    ({"fft_tile": 8192}, "fft_tile"),
    ({"fft_tile": 100}, "fft_tile"),
    ({"gemm_max_level": 4096}, "gemm_max_level"),
    ({"solver": 4}, "solver"),
    ({"solver": -1}, "solver"),
])
def test_invalid_tuning_rejected(tune, msg):
    with pytest.raises(ftoep.FtoepError) as ei:
        ftoep.ftoep_create([_spec()], tune, 0)
    assert ei.value.status == ftoep.FTOEP_EINVAL and msg in str(ei.value)


def test_invalid_problem_in_a_batch_names_its_index():
    with pytest.raises(ftoep.FtoepError) as ei:
        ftoep.ftoep_create([_spec(), _spec(), _spec(kind=1, gamma=0.7)], None, 0)
    assert ei.value.status == ftoep.FTOEP_EINVAL and "problem 2" in str(ei.value)


def test_autotune_validates_before_timing():
    with pytest.raises(ftoep.FtoepError) as ei:
        ftoep.ftoep_autotune([_spec(gamma=1.5)], stream=0)
    assert ei.value.status == ftoep.FTOEP_EINVAL


def test_tuning_key_buckets_and_cache_roundtrip(tmp_path, monkeypatch):
    """The autotuner's cache key groups problems by (ceil log2 N, ceil log2 (M+1), precision,
    kind, space) and the device; a cached entry is returned without running the autotuner."""
    import json
    from paper_1710_11593_gb300 import ftoep
    a = [ftoep.ProblemSpec(0, 0.5, 1000, 63, 1, 1), ftoep.ProblemSpec(1, 1.5, 1024, 60, 1, 1)]
    b = [ftoep.ProblemSpec(1, 1.7, 600, 50, 1, 1), ftoep.ProblemSpec(0, 0.2, 513, 33, 1, 1)]
    c = [ftoep.ProblemSpec(0, 0.5, 1025, 63, 1, 1), ftoep.ProblemSpec(1, 1.5, 1024, 60, 1, 1)]
    assert ftoep.tuning_key(a, "X") == ftoep.tuning_key(b, "X")
    assert ftoep.tuning_key(a, "X") != ftoep.tuning_key(c, "X")
    assert ftoep.tuning_key(a, "X") != ftoep.tuning_key(a, "Y")
    path = tmp_path / "t.json"
    key = ftoep.tuning_key(a, "")
    want = {"leaf": 0, "fft_tile": 2048, "gemm_max_level": 0, "scheduler": 2, "streams": 8, "solver": 2}
    path.write_text(json.dumps({key: want}))
    monkeypatch.setattr(ftoep, "ftoep_autotune", lambda *x, **k: (_ for _ in ()).throw(AssertionError("ran")))
    import sys
    monkeypatch.setitem(sys.modules, "torch", None)  # no device name: the key of the stored entry
    got, hit = ftoep.autotune_cached(a, path=str(path))
    assert hit and got == want


@pytest.mark.parametrize("kw", [dict(gamma=1.2), dict(gamma=0.0), dict(N=1), dict(tol=0.0), dict(maxit=0),
                                dict(T=-1.0)])
def test_two_sided_cg_validates_before_any_device_work(kw):
    """Argument checks of ftoep_two_sided_cg return FTOEP_EINVAL before touching CUDA."""
    import numpy as np
    from paper_1710_11593_gb300 import ftoep
    args = dict(gamma=0.5, T=1.0, N=10, tol=1e-10, maxit=10)
    args.update(kw)
    f = np.ones(max(1, args["N"] - 1))
    u = np.zeros_like(f)
    lib = ftoep.load()
    import ctypes
    rc = lib.ftoep_two_sided_cg(args["gamma"], args["T"], args["N"], f.ctypes.data, u.ctypes.data, args["tol"],
                                args["maxit"], None, None, None)
    assert rc == ftoep.FTOEP_EINVAL


@pytest.mark.parametrize("kw", [dict(scheme=1), dict(scheme=2, gamma=1.5), dict(scheme=3, gamma=0.5), dict(N=0),
                                dict(M=0), dict(T=0.0), dict(L=-1.0), dict(precision=2)])
def test_advection_sweep_validates_before_any_device_work(kw):
    """Argument checks of ftoep_advection_sweep return FTOEP_EINVAL before touching CUDA."""
    import numpy as np
    from paper_1710_11593_gb300 import ftoep
    args = dict(scheme=2, gamma=0.5, T=1.0, L=1.0, N=8, M=4, precision=0)
    args.update(kw)
    f = np.ones(max(1, args["M"] * args["N"]))
    u = np.zeros_like(f)
    lib = ftoep.load()
    rc = lib.ftoep_advection_sweep(args["scheme"], args["gamma"], args["T"], args["L"], args["N"], args["M"],
                                   f.ctypes.data, None, None, u.ctypes.data, args["precision"], None)
    assert rc == ftoep.FTOEP_EINVAL


def test_gmres_validates_its_arguments():
    """ftoep_gmres without a plan returns FTOEP_EINVAL (no device work)."""
    import numpy as np
    from paper_1710_11593_gb300 import ftoep
    f = np.ones(8)
    u = np.zeros(8)
    lib = ftoep.load()
    assert lib.ftoep_gmres(None, 0, f.ctypes.data, u.ctypes.data, 10, 1e-10, 10, None, None) == ftoep.FTOEP_EINVAL


def test_shipped_tuning_table_is_valid():
    """The autotuner's table shipped with the package: every entry is a valid tuning for
    ftoep_create and is keyed like tuning_key (device | buckets)."""
    import json
    from paper_1710_11593_gb300 import ftoep
    with open(ftoep.SHIPPED_TUNING) as fh:
        table = json.load(fh)
    assert table
    for key, entry in table.items():
        assert "|" in key and key.split("|")[0]
        t = {k: int(entry.get(k, 0)) for k in ftoep.TUNING_FIELDS}
        assert t["fft_tile"] in (0, 1024, 2048, 4096) and t["scheduler"] in (0, 1, 2)
        assert 0 <= t["streams"] <= 8 and t["solver"] in (0, 1, 3)
