"""The C ABI library builds, loads and exports every entry point that
include/tdbem.h declares, and the Python binding covers exactly those (no
compute calls: this runs without a GPU)."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tdbem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tdbem_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("tdbem_create", "tdbem_destroy", "tdbem_set_mesh", "tdbem_set_bc", "tdbem_set_known",
              "tdbem_set_incident_plane", "tdbem_prepare", "tdbem_step", "tdbem_get_solution",
              "tdbem_get_stats", "tdbem_last_error"):
        assert n in names


def test_library_builds_and_exports_every_symbol():
    from paper_2111_05205_gb300 import abi, build
    path = build.build()
    assert os.path.exists(path)
    L = abi.lib()
    for n in _declared():
        assert hasattr(L, n), n


def test_binding_matches_header():
    from paper_2111_05205_gb300 import abi
    assert sorted(abi.SIGNATURES) == _declared()
    for n in _declared():
        assert callable(getattr(abi, n))


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2111_05205_gb300 import abi, build
    monkeypatch.setattr(build, "LIB", str(tmp_path / "nope.so"))
    monkeypatch.setattr(abi, "_lib", None)
    with pytest.raises(RuntimeError):
        abi.lib()


def test_null_context_is_an_error_not_a_crash():
    from paper_2111_05205_gb300 import abi
    L = abi.lib()
    assert L.tdbem_prepare(None) == -1
    assert L.tdbem_step(None, 1) == -1
    assert L.tdbem_last_error(None) == b"null context"
