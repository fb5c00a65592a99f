"""Failure detection on the GPU without faulting it: a sweep hand-off wait that runs out
returns RTE_ERR_DEP_TIMEOUT (the kernel finishes; the wait limit is made small on purpose),
non-finite data give RTE_ERR_NAN, and a host-injected zero Galerkin pivot gives
RTE_ERR_SINGULAR.  After each failure the handle (and the CUDA context) stays usable: the same
call with sane settings reproduces the oracle."""
import numpy as np
import pytest

import workloads as W
from tests.helpers import gpu_handle, oracle_disc, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    from paper_2603_25233_gb300 import _lib as L
    return L


def test_sweep_wait_that_runs_out_reports_timeout_and_the_handle_recovers():
    """70 rows = 3 bands of 32: the second and third bands wait on the band below.  With one
    poll allowed, the first wait gives up long before the producing warp has finished 4
    columns, so the flag is set; the call returns RTE_ERR_DEP_TIMEOUT and does not hang."""
    from oracle.transport import DirectSweeper
    L = _lib()
    spec = W.random_small(40, 70, n_theta=8, n_omz=2, seed=2)
    d = oracle_disc(spec)
    S = np.abs(np.random.default_rng(3).standard_normal(d.ndof))
    angles = np.arange(d.n_angles)
    with gpu_handle(spec) as h:
        src = torch.tensor(S, dtype=torch.float32, device="cuda")
        psi = torch.empty(len(angles) * d.ndof, dtype=torch.float32, device="cuda")
        h.set_wait_limit(1)
        with pytest.raises(L.RteError) as ei:
            h.sweep(angles, src, L.RTE_FP32, psi_out=psi)
        assert ei.value.code == L.RTE_ERR_DEP_TIMEOUT
        with pytest.raises(L.RteError) as ei:
            h.si_dsa_solve(mode="fr", sweep_precision="fp32", eps_si=1e-8, max_outer=5)
        assert ei.value.code == L.RTE_ERR_DEP_TIMEOUT
        h.set_wait_limit(0)
        h.sweep(angles, src, L.RTE_FP32, psi_out=psi)
        P = psi.double().cpu().numpy().reshape(len(angles), d.ndof)
    sw = DirectSweeper(d)
    for a, j in enumerate(angles):
        assert rel_l2(P[a], sw.sweep(j, S)) < 2e-5


@pytest.mark.parametrize("mode", ["fr", "lr"])
def test_non_finite_initial_flux_reports_nan(mode):
    L = _lib()
    spec = W.random_small(9, 7, n_theta=8, n_omz=2, seed=4)
    with gpu_handle(spec) as h:
        phi = torch.full((h.n_dof,), float("nan"), dtype=torch.float64, device="cuda")
        with pytest.raises(L.RteError) as ei:
            h.si_dsa_solve(mode=mode, sweep_precision="fp64", eps_si=1e-10, eps_res=1e-11, eps_diff=1e-11,
                           max_outer=50, phi=phi)
        assert ei.value.code == L.RTE_ERR_NAN
        phi2, st = h.si_dsa_solve(mode=mode, sweep_precision="fp64", eps_si=1e-10, eps_res=1e-11, eps_diff=1e-11,
                                  max_outer=200)
        assert st["converged"] == 1 and bool(torch.isfinite(phi2).all())


def test_injected_zero_galerkin_pivot_reports_singular_once():
    from oracle import lowrank
    L = _lib()
    spec = W.random_small(8, 6, n_theta=16, n_omz=2, seed=5)
    d = oracle_disc(spec)
    opts = dict(eps_res=1e-9, eps_diff=1e-9, p=1, q=4, seed=7)
    ref = lowrank.lowrank_si(d, np.zeros(d.ndof), 1, opts)
    with gpu_handle(spec) as h:
        h.inject_failure(L.RTE_ERR_SINGULAR)
        with pytest.raises(L.RteError) as ei:
            h.si_dsa_solve(mode="lr", sweep_precision="fp64", max_outer=1, use_dsa=0, eps_si=0.0, truncate=0, **opts)
        assert ei.value.code == L.RTE_ERR_SINGULAR
        phi, st = h.si_dsa_solve(mode="lr", sweep_precision="fp64", max_outer=1, use_dsa=0, eps_si=0.0, truncate=0,
                                 **opts)
    assert st["final_rank"] == ref["rank"] and st["total_inner"] == ref["stats"]["inner"]
    assert rel_l2(phi.cpu().numpy(), ref["phi"]) < 1e-11
