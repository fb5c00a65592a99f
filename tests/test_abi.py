"""The C-ABI library builds, loads and exports every entry point include/rte.h declares (CPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "rte.h")).read()
    return re.findall(r"^\s*(?:int|void|const char\*)\s+(rte_\w+)\s*\(", txt, re.M)


def test_library_exports_every_declared_symbol():
    from paper_2603_25233_gb300 import build as B
    B.build()
    lib = ctypes.CDLL(B.LIB)
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_signatures_cover_header():
    from paper_2603_25233_gb300 import _lib as L
    assert set(_declared()) <= set(L.SIGNATURES)


def test_default_opts_follow_paper_defaults():
    from paper_2603_25233_gb300 import _lib as L
    lib = L.load()
    o = L.RteOpts()
    lib.rte_default_opts(ctypes.byref(o))
    assert (o.eps_si, o.eps_res, o.eps_diff, o.eps_svd, o.eps_mgs) == (1e-6, 1e-7, 1e-7, 1e-8, 1e-10)
    assert (o.p, o.q, o.m_max, o.dsa_tol) == (1, 8, 4, 1e-12)


def test_setup_rejects_bad_arguments_without_touching_the_gpu():
    from paper_2603_25233_gb300 import _lib as L
    lib = L.load()
    p = L.RteProblem()
    p.nx, p.ny, p.n_theta, p.n_omz = 4, 4, 6, 2     # n_theta not a multiple of 4
    p.x0, p.x1, p.y0, p.y1 = 0, 1, 0, 1
    h = ctypes.c_void_p()
    rc = lib.rte_setup(ctypes.byref(p), None, ctypes.byref(h))
    assert rc == L.RTE_ERR_ARG and not h.value
    assert b"multiple of 4" in lib.rte_last_error()
    assert lib.rte_destroy(None) == 0


def test_product_path_fails_loudly_without_library(tmp_path):
    from paper_2603_25233_gb300 import _lib as L
    with pytest.raises(OSError):
        L._lib_backup = L._lib
        try:
            L._lib = None
            L.load(str(tmp_path / "missing.so"))
        finally:
            L._lib = L._lib_backup


def test_static_dsa_solve_rejects_meshes_beyond_its_scratch():
    """Size checks come before any CUDA call, so this runs without a GPU."""
    from paper_2603_25233_gb300 import _lib as L
    lib = L.load()
    dummy = ctypes.c_void_p(16)
    rc = lib.rte_dsa_solve_static(200, 100, 0.0, 1.0, 0.0, 1.0, dummy, dummy, dummy, dummy, 1e-8, 10, None, None)
    assert rc == L.RTE_ERR_ARG
    assert b"16384 cells" in lib.rte_last_error()


def _problem(L, nx=4, ny=3):
    p = L.RteProblem()
    p.nx, p.ny, p.n_theta, p.n_omz = nx, ny, 8, 2
    p.x0, p.x1, p.y0, p.y1 = 0.0, 1.0, 0.0, 1.0
    return p


def test_setup_rejects_non_finite_materials_and_bad_gaussians_without_touching_the_gpu():
    """Host-injected non-finite data: a NaN cross section, and Gaussian sources with a
    non-positive or non-finite exponent, are refused by rte_setup before any device work."""
    import numpy as np
    from paper_2603_25233_gb300 import _lib as L
    lib = L.load()
    dp = ctypes.POINTER(ctypes.c_double)
    st = np.ones(12)
    ss = np.full(12, 0.5)
    for bad in ("sig_t_nan", "sig_s_nan", "sig_t_inf"):
        p = _problem(L)
        a_t, a_s = st.copy(), ss.copy()
        if bad == "sig_t_nan":
            a_t[5] = np.nan
        elif bad == "sig_s_nan":
            a_s[2] = np.nan
        else:
            a_t[0] = np.inf
        p.sig_t, p.sig_s = a_t.ctypes.data_as(dp), a_s.ctypes.data_as(dp)
        h = ctypes.c_void_p()
        assert lib.rte_setup(ctypes.byref(p), None, ctypes.byref(h)) == L.RTE_ERR_ARG and not h.value, bad
    for g in ((0.0, 0.0, 0.0, 1.0), (0.0, 0.0, -1.0, 1.0), (0.0, 0.0, np.nan, 1.0), (np.inf, 0.0, 1.0, 1.0)):
        p = _problem(L)
        p.sig_t, p.sig_s = st.ctypes.data_as(dp), ss.ctypes.data_as(dp)
        ga = np.array(g, dtype=np.float64)
        p.n_gauss, p.q_gauss = 1, ga.ctypes.data_as(dp)
        h = ctypes.c_void_p()
        assert lib.rte_setup(ctypes.byref(p), None, ctypes.byref(h)) == L.RTE_ERR_ARG and not h.value, g
        assert b"Gaussian" in lib.rte_last_error()


def test_failure_hooks_reject_bad_arguments():
    from paper_2603_25233_gb300 import _lib as L
    lib = L.load()
    assert lib.rte_set_wait_limit(None, 10) == L.RTE_ERR_ARG
    assert lib.rte_inject_failure(None, L.RTE_ERR_SINGULAR) == L.RTE_ERR_ARG


def test_sweep_autotuner_calls_reject_bad_arguments():
    from paper_2603_25233_gb300 import _lib as L
    lib = L.load()
    c = L.RteSweepConfig()
    assert lib.rte_sweep_tune(None, L.RTE_FP32, 8, 1, ctypes.byref(c)) == L.RTE_ERR_ARG
    assert lib.rte_sweep_set_config(None, L.RTE_FP32, 8, 1, None) == L.RTE_ERR_ARG
    assert lib.rte_sweep_get_config(None, L.RTE_FP64, 8, 0, ctypes.byref(c)) == L.RTE_ERR_ARG


def test_lowrank_state_rejects_a_null_handle():
    from paper_2603_25233_gb300 import _lib as L
    lib = L.load()
    assert lib.rte_get_lowrank_state(None, None, None, None, None, None, None) == L.RTE_ERR_ARG
