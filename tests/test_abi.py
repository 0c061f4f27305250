"""The C ABI library builds, loads and exports every entry point declared in
include/ftoep.h (no GPU needed: nothing is called)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*ftoep_status\s+(ftoep_\w+)\s*\(", src, re.M))
    return names


def test_library_exports_all_declared_symbols():
    from paper_1710_11593_gb300 import build
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(ftoep_\w+)", out))
    declared = _declared()
    assert declared, "no declarations found"
    missing = declared - exported
    assert not missing, f"declared but not exported: {missing}"


def test_binding_loads_and_binds_every_symbol():
    from paper_1710_11593_gb300 import ftoep
    lib = ftoep.load()
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(ftoep.EXPORTS) <= _declared()


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1710_11593_gb300 import ftoep
    with pytest.raises(ftoep.FtoepError):
        ftoep.load.__wrapped__(str(tmp_path / "missing.so")) if hasattr(ftoep.load, "__wrapped__") else \
            _load_fresh(ftoep, str(tmp_path / "missing.so"))


def _load_fresh(ftoep, path):
    saved = ftoep._lib
    ftoep._lib = None
    try:
        return ftoep.load(path)
    finally:
        ftoep._lib = saved
