"""The C ABI library builds for sm_103a, loads on a machine without a GPU,
and exports every entry point include/vlbm.h declares (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "vlbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vlbm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("vlbm_create_hierarchy", "vlbm_set_state", "vlbm_advance", "vlbm_regrid", "vlbm_get_conserved"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2609_35529_b300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2609_35529_b300 import vlbm
    monkeypatch.setattr(vlbm, "_lib", None)
    monkeypatch.setattr(vlbm, "LIB_PATH", str(tmp_path / "missing.so"))
    import pytest
    with pytest.raises(RuntimeError):
        vlbm.lib()
