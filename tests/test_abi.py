"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function declared in include/pierce.h; the Python binding covers them all."""
import ctypes
import os
import re

import pytest

from paper_2609_24513_gb300 import _build, pierce

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pierce.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pj_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("pj_create", "pj_destroy", "pj_load_meshes", "pj_build_bvh",
              "pj_join_intersects", "pj_free_pairs", "pj_get_counters", "pj_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    assert set(_declared()) <= set(pierce.SIGNATURES)


def test_struct_sizes_match_header_layout():
    assert ctypes.sizeof(pierce.pj_config) == 32
    assert ctypes.sizeof(pierce.pj_join_opts) == 48
    assert ctypes.sizeof(pierce.pj_pairs) == 88
    assert ctypes.sizeof(pierce.pj_counters) == 16 * 8


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(pierce, "_lib", None)
    monkeypatch.setattr(pierce._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        pierce.load()
