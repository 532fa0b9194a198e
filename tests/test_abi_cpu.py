"""The C ABI library loads without a GPU and exports every function include/acse.h declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "acse.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(acse_[A-Za-z0-9_]+)\s*\(", src)))


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for want in ("acse_create", "acse_destroy", "acse_energy", "acse_residual", "acse_step",
                 "acse_residual_backward", "acse_strerror"):
        assert want in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2604_02550_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    L = _lib.lib()
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    assert set(_declared()) == set(_lib.EXPORTS)
    assert "sm_103a" in _lib.version()
    assert _lib.strerror(-9).startswith("r exceeds")


def test_binding_refuses_to_run_without_library(monkeypatch, tmp_path):
    from paper_2604_02550_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        _lib.lib()
