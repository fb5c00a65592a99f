"""The allocation-free DSA solve (rte_dsa_solve_static) against the handle-based one.

rte_dsa_solve_static serves callers that cannot allocate device memory; its scratch is a fixed
device array shared by all calls.  Two calls in a row, with different right-hand sides, must
each agree with rte_dsa_solve on the same system within the tolerance of the DSA tests.  The
static solve preconditions with block Jacobi only (the vertex multigrid of the handle-based
solve needs a hierarchy built per problem), so only the solutions are compared, not the
iteration counts.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _static_solve(lib, spec, sig_t, sig_s, rhs, tol, max_iter):
    x = torch.full_like(rhs, float("nan"))
    it = ctypes.c_int(-1)
    rc = lib.rte_dsa_solve_static(spec.nx, spec.ny, spec.x0, spec.x1, spec.y0, spec.y1,
                                  ctypes.c_void_p(sig_t.data_ptr()), ctypes.c_void_p(sig_s.data_ptr()),
                                  ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                  tol, max_iter, ctypes.byref(it),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, x, it.value


def test_static_dsa_solve_matches_handle_solve_twice():
    from paper_2603_25233_gb300 import _lib as L
    from paper_2603_25233_gb300.api import Handle
    lib = L.load()
    spec = W.random_small(60, 45, n_theta=8, n_omz=2, seed=21, sig_range=(0.5, 50.0), ratio_range=(0.5, 0.999))
    sig_t = torch.tensor(spec.sig_t, device="cuda")
    sig_s = torch.tensor(spec.sig_s, device="cuda")
    rng = np.random.default_rng(3)
    tol, max_iter = 1e-12, 20000
    with Handle(spec) as h:
        for call in range(2):
            rhs = torch.tensor(rng.standard_normal(h.n_dof), device="cuda")
            x_ref, it_ref = h.dsa_solve(rhs, tol=tol, max_iter=max_iter)
            rc, x, it = _static_solve(lib, spec, sig_t, sig_s, rhs, tol, max_iter)
            torch.cuda.synchronize()
            assert rc == L.RTE_OK, lib.rte_last_error().decode()
            assert 0 < it_ref <= it < max_iter
            err = float(torch.linalg.vector_norm(x - x_ref) / torch.linalg.vector_norm(x_ref))
            assert err < 1e-9, (call, err)
