"""The C-ABI library builds for sm_103a and exports every entry point declared in include/stst.h (no GPU needed)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "stst.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(stst_[a-z0-9_]+)\s*\(", txt)))


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="CUDA toolkit absent")
def test_library_builds_and_exports_every_declared_symbol():
    from paper_2311_18461_gb300 import build
    path = build.build()
    L = ctypes.CDLL(path)
    names = _declared()
    assert "stst_pcg_solve" in names and "stst_apply_prec" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(monkeypatch):
    import paper_2311_18461_gb300._lib as B
    monkeypatch.setattr(B, "library_path", "/nonexistent/libstst.so")
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(RuntimeError):
        B.lib()


def test_binding_names_match_header():
    import paper_2311_18461_gb300 as P
    for n in _declared():
        assert hasattr(P, n), n
