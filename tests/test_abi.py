"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/kmp.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "kmp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(kmp_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2105_02022_gb300 import _build

    path = _build.build_kmp()
    return ctypes.CDLL(path), path


def test_every_declared_symbol_exported(lib):
    L, path = lib
    names = declared()
    assert len(names) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (kmp_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(L, n)


def test_config_roundtrip_without_gpu(lib):
    from paper_2105_02022_gb300 import kmp

    c = kmp.config()
    assert (c.C, c.lp_rounds, c.refine_rounds, c.subrounds) == (160, 5, 5, 8)
    import oracle

    oc = oracle.config()
    for name, _ in kmp.Config._fields_:
        assert getattr(c, name) == getattr(oc, name), name


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2105_02022_gb300 import _build, kmp

    monkeypatch.setattr(_build, "lib_path", lambda: str(tmp_path / "missing.so"))
    monkeypatch.setattr(kmp, "_LIB", None)
    with pytest.raises(ImportError):
        kmp.load()
