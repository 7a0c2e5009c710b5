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


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="CUDA toolkit absent")
def test_host_side_argument_checks_need_no_gpu():
    """The calls that reject arguments before any CUDA call return the documented status codes; the
    process-wide tuning switches are restored to their defaults (autotune 1, time solver 0, fused 0)."""
    from paper_2311_18461_gb300 import build
    L = ctypes.CDLL(build.build())
    ERR_ARG, ERR_HANDLE = -1, -2
    try:
        for mode in (0, 1, 132, 12, 14, 22, 44):
            assert L.stst_set_autotune(mode) == 0, mode
        for mode in (-1, 2, 15, 52, 99, 131):
            assert L.stst_set_autotune(mode) == ERR_ARG, mode
        for mode in (0, 1, 2, 11, 14):
            assert L.stst_set_fused_transforms(mode) == 0, mode
        for mode in (-1, 3, 10, 15):
            assert L.stst_set_fused_transforms(mode) == ERR_ARG, mode
        for mode in (0, 1, 2):
            assert L.stst_set_time_solver(mode) == 0, mode
        for mode in (-1, 3):
            assert L.stst_set_time_solver(mode) == ERR_ARG, mode
        for mode in (0, 1, 2, 3):
            assert L.stst_set_pencil(mode) == 0, mode
        for mode in (-1, 4):
            assert L.stst_set_pencil(mode) == ERR_ARG, mode
        for mode in (0, 1, 2):
            assert L.stst_set_tensor_products(mode) == 0, mode
        for mode in (-1, 3):
            assert L.stst_set_tensor_products(mode) == ERR_ARG, mode
        for mode in (0, 1):
            assert L.stst_set_fused_matvec(mode) == 0, mode
        for mode in (-1, 2):
            assert L.stst_set_fused_matvec(mode) == ERR_ARG, mode
    finally:
        L.stst_set_autotune(1)
        L.stst_set_time_solver(0)
        L.stst_set_fused_transforms(0)
        L.stst_set_pencil(0)
        L.stst_set_tensor_products(0)
        L.stst_set_fused_matvec(0)
    n = ctypes.c_longlong()
    assert L.stst_sizes(None, ctypes.byref(n), None) == ERR_HANDLE
    assert L.stst_pcg_graph_info(None, None, None) == ERR_HANDLE
    assert L.stst_build_fd(None) == ERR_HANDLE
    assert L.stst_set_potential(None, 0, None) == ERR_HANDLE
    assert L.stst_pencil_info(None, None) == ERR_HANDLE
    assert L.stst_fused_transforms_split(None, None, None) == ERR_HANDLE
    assert L.stst_tensor_products_info(None, None) == ERR_HANDLE
    assert L.stst_set_geometry(None, None, None) == ERR_HANDLE
    assert L.stst_geometry_info(None, None, None, None) == ERR_HANDLE
    # the persistent solver: counts, arrays and cluster sizes are checked before any handle or CUDA call
    hs = (ctypes.c_void_p * 1)(None)
    vp = (ctypes.c_void_p * 1)(None)
    L.stst_persistent_solve.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    ps = L.stst_persistent_solve
    assert ps(0, hs, vp, vp, 1e-8, 10, 8, None, None, None, None) == ERR_ARG
    assert ps(1, None, vp, vp, 1e-8, 10, 8, None, None, None, None) == ERR_ARG
    assert ps(1, hs, vp, vp, -1.0, 10, 8, None, None, None, None) == ERR_ARG
    assert ps(1, hs, vp, vp, 1e-8, -1, 8, None, None, None, None) == ERR_ARG
    for bad_cluster in (3, 32, -1):
        assert ps(1, hs, vp, vp, 1e-8, 10, bad_cluster, None, None, None, None) == ERR_ARG, bad_cluster
    assert ps(1, hs, vp, vp, 1e-8, 10, 8, None, None, None, None) == ERR_HANDLE
    out = ctypes.c_int()
    bad = [(0, 4, 1.0, 2), (9, 4, 1.0, 2), (2, 0, 1.0, 2), (2, 4, 0.0, 2), (2, 4, -1.0, 1), (2, 4, 1.0, 3),
           (1, 1, 1.0, 2)]  # the last leaves no function after dropping both ends
    for p, n_el, length, bc in bad:
        assert L.stst_assemble_1d(p, n_el, ctypes.c_double(length), bc, None, None, None, None, None, None,
                                  ctypes.byref(out), None) == ERR_ARG, (p, n_el, length, bc)
    L.stst_strerror.restype = ctypes.c_char_p
    texts = {s: L.stst_strerror(s).decode() for s in (0, 1, 2, 3, 4, -1, -2, -3, -4, -5)}
    assert len(set(texts.values())) == len(texts) and "unknown" not in " ".join(texts.values())
    assert L.stst_strerror(77).decode() == "unknown status"
