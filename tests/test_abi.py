"""The C ABI library loads and exports every function include/polydg.h declares (no GPU)."""
import os
import re

from conftest import ROOT


def header_functions():
    text = open(os.path.join(ROOT, "include", "polydg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


def ensure_built():
    import paper_2512_19536_gb300 as pd
    if not os.path.exists(pd.LIB_PATH):
        from paper_2512_19536_gb300.build import build
        build()
    return pd


def test_library_exports_every_header_function():
    pd = ensure_built()
    L = pd.load()
    declared = header_functions()
    assert len(declared) >= 16
    for name in declared:
        assert hasattr(L, name), name
    assert sorted(pd.EXPORTS) == declared


def test_last_error_starts_empty():
    pd = ensure_built()
    assert pd.load().polydg_last_error() in (b"",) or isinstance(pd.load().polydg_last_error(), bytes)


def test_binding_refuses_missing_library(tmp_path, monkeypatch):
    import paper_2512_19536_gb300._native as nat
    monkeypatch.setattr(nat, "_lib", None)
    monkeypatch.setattr(nat, "LIB_PATH", str(tmp_path / "missing.so"))
    try:
        nat.load()
    except RuntimeError as e:
        assert "missing" in str(e)
    else:
        raise AssertionError("load() must fail without the library")
