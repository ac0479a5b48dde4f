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
    assert ctypes.sizeof(pierce.pj_join_opts) == 56
    assert ctypes.sizeof(pierce.pj_pairs) == 96
    assert ctypes.sizeof(pierce.pj_counters) == 20 * 8
    assert ctypes.sizeof(pierce.pj_query) == 40
    assert ctypes.sizeof(pierce.pj_query_stats) == 80


_STRUCTS = ("pj_config", "pj_bvh_params", "pj_join_opts", "pj_pairs", "pj_counters",
            "pj_dataset_info", "pj_tune_space", "pj_tune_entry", "pj_query", "pj_query_stats",
            "pj_estimate", "pj_dsjoin_opts", "pj_dsjoin_stats", "pj_host_meshes",
            "pj_tiled_opts", "pj_tiled_stats")


def test_struct_layout_matches_the_c_compiler(tmp_path):
    """Every struct's size and every field's offset as gcc lays out the
    header, against the ctypes mirror."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pierce.h"',
             'int main(void) {']
    for st in _STRUCTS:
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (st, st))
        for f, _ in getattr(pierce, st)._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (st, f, st, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for st in _STRUCTS:
        cls = getattr(pierce, st)
        assert int(out[st]) == ctypes.sizeof(cls), st
        for f, _ in cls._fields_:
            assert int(out["%s.%s" % (st, f)]) == getattr(cls, f).offset, (st, f)


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(pierce, "_lib", None)
    monkeypatch.setattr(pierce._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        pierce.load()


def test_no_cpu_fallback_without_a_gpu():
    """With the library present but no CUDA device, creating a context fails
    with PJ_ERR_CUDA: nothing runs on the host instead."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pierce.PierceError) as e:
        pierce.pj_create(0)
    assert "PJ_ERR_CUDA" in str(e.value)
    assert pierce.pj_last_error(None) == "null context"
