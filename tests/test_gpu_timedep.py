"""GPU parity of the backward-Euler step (rte_be_step, Sec. 3.7) with the oracle's coupled
solve of the step and its SI-DSA: single steps from an anisotropic random psi^n, marching over
several steps, FP32 sweeps, the homogeneous closed form, and the handle's steady problem left
unchanged."""
import math

import numpy as np
import pytest

import workloads as W
from tests.helpers import gpu_handle, oracle_disc, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _spec(nx, ny, seed, **kw):
    return W.random_small(nx, ny, n_theta=8, n_omz=2, seed=seed, inflow=(0.3, 0.1, 0.2, 0.4),
                          box=(0.0, 1.3, -0.2, 0.9), **kw)


def _psi0(d, seed):
    rng = np.random.default_rng(seed)
    return np.abs(rng.standard_normal((d.ndof, d.n_angles)))          # [N_x, N_Omega]


def _dev(psi):                                                      # to ordinate-major device
    return torch.tensor(np.ascontiguousarray(psi.T).ravel(), device="cuda")


def _host(psi_dev, d):
    return psi_dev.cpu().numpy().reshape(d.n_angles, d.ndof).T


# a mesh below one band (warp kernel) also against the coupled solve of the step; meshes of
# several bands (band kernel, ragged) against the oracle's SI-DSA of the step, which the
# oracle's pins tie to the coupled solve (the coupled LU takes minutes there)
@pytest.mark.parametrize("shape,dt,coupled", [((7, 37), 0.05, True), ((40, 33), 0.5, False), ((33, 64), 3.0, False)])
def test_step_matches_oracle_si_iterations(shape, dt, coupled):
    from oracle import timedep
    spec = _spec(*shape, seed=11, ratio_range=(0.5, 0.99))
    d = oracle_disc(spec)
    psi0 = _psi0(d, 12)
    ref = timedep.be_si_dsa(spec, psi0, dt, eps_si=1e-11, max_iter=500)
    with gpu_handle(spec) as h:
        phi, psi, st = h.be_step(dt, _dev(psi0), mode="fr", sweep_precision="fp64", eps_si=1e-11, max_outer=500,
                                 dsa_tol=1e-12)
    assert st["converged"] == 1 and st["outer_iters"] == ref["iters"]
    assert rel_l2(phi.cpu().numpy(), ref["phi"]) < 1e-10
    assert rel_l2(_host(psi, d).ravel(), ref["psi"].ravel()) < 1e-10
    if coupled:
        phi_c, psi_c = timedep.be_coupled_solve(d, psi0, dt)
        assert rel_l2(phi.cpu().numpy(), phi_c) < 1e-9
        assert rel_l2(_host(psi, d).ravel(), psi_c.ravel()) < 1e-9


def test_marching_three_steps_matches_oracle():
    from oracle import timedep
    spec = _spec(12, 10, seed=13)
    d = oracle_disc(spec)
    psi0 = _psi0(d, 14)
    dt = 0.2
    ref = timedep.be_march(spec, psi0, dt, 3)
    with gpu_handle(spec) as h:
        psi = _dev(psi0)
        phi = torch.zeros(h.n_dof, dtype=torch.float64, device="cuda")
        for k in range(3):
            phi, psi, st = h.be_step(dt, psi, phi=phi, psi_next=psi, mode="fr", sweep_precision="fp64",
                                     eps_si=1e-12, max_outer=500, dsa_tol=1e-12)
            assert st["converged"] == 1
            assert rel_l2(phi.cpu().numpy(), ref[k][0]) < 1e-9
            assert rel_l2(_host(psi, d).ravel(), ref[k][1].ravel()) < 1e-9


def test_fp32_sweeps_within_single_precision():
    from oracle import timedep
    spec = _spec(40, 33, seed=15)
    d = oracle_disc(spec)
    psi0 = _psi0(d, 16)
    phi_c = timedep.be_si_dsa(spec, psi0, 0.5, eps_si=1e-12, max_iter=500)["phi"]
    with gpu_handle(spec) as h:
        phi, _, st = h.be_step(0.5, _dev(psi0), mode="fr", sweep_precision="fp32", sweep_refine=0, eps_si=1e-7,
                               max_outer=500)
    assert st["converged"] == 1
    assert rel_l2(phi.cpu().numpy(), phi_c) < 1e-5


def test_homogeneous_closed_form_and_steady_problem_restored():
    """Constant medium, psi^0 = c0, inflow at the exact next value c1 = (c0/dt + q)/(1/dt +
    sigma_a): the step returns the constant c1; afterwards the handle's steady solve still
    matches the oracle's steady solution (the step's sigma_t shift is undone)."""
    sig_t, sig_s, q, dt, c0 = 2.0, 1.5, 1.0, 0.3, 0.2
    c1 = (c0 / dt + q) / (1.0 / dt + sig_t - sig_s)
    spec = W.infinite_medium(9, 40, sig_t, sig_s, q, n_theta=8, n_omz=2, box=(0.0, 1.3, -0.2, 0.7))
    spec.inflow = (c1,) * 4
    d = oracle_disc(spec)
    unit = math.sqrt(d.hx * d.hy)
    const = np.zeros(d.ndof)
    const[0::4] = unit
    with gpu_handle(spec) as h:
        psi0 = _dev(np.tile((c0 * const)[:, None], (1, d.n_angles)))
        phi, psi, st = h.be_step(dt, psi0, mode="fr", sweep_precision="fp64", eps_si=1e-14, max_outer=500,
                                 dsa_tol=1e-13)
        assert np.abs(phi.cpu().numpy() - c1 * const).max() < 1e-12
        assert np.abs(_host(psi, d) - (c1 * const)[:, None]).max() < 1e-12
        phi_s, st_s = h.si_dsa_solve(mode="fr", sweep_precision="fp64", eps_si=1e-13, max_outer=500)
        from oracle import si_dsa
        ref = si_dsa.fr_si_dsa(d, eps_si=1e-13, max_iter=500)["phi"]
        assert rel_l2(phi_s.cpu().numpy(), ref) < 1e-10


def test_step_rejects_bad_arguments():
    from paper_2603_25233_gb300._lib import RteError
    spec = _spec(6, 5, seed=17)
    with gpu_handle(spec) as h:
        psi0 = torch.zeros(h.n_angles * h.n_dof, dtype=torch.float64, device="cuda")
        for kw in (dict(mode=7), dict(sweep_precision="fp32", sweep_refine=1)):
            with pytest.raises(RteError):
                h.be_step(0.1, psi0, **kw)
        for dt in (0.0, -1.0, float("inf")):
            with pytest.raises(RteError):
                h.be_step(dt, psi0)


def _twin_symmetric(d, psi):
    from oracle.lowrank import twin_map
    tw = twin_map(d)
    return 0.5 * (psi + psi[:, tw])


@pytest.mark.parametrize("basis", ["fp64", "dw"])
def test_lowrank_step_matches_oracle(basis):
    """The low-rank step (Alg. 1 on the step's steady problem, the time source in the sampled
    sweeps, the bordered Galerkin right-hand sides and the candidate residuals) against the
    oracle's: outer and inner iteration counts, phi, and psi^{n+1} = X C."""
    from oracle import timedep
    spec = _spec(8, 6, seed=21)
    d = oracle_disc(spec)
    psi0 = _twin_symmetric(d, _psi0(d, 22))
    dt = 0.3
    opts = dict(eps_si=1e-9, eps_res=1e-10, eps_diff=1e-10, p=1, q=4, seed=11)
    ref = timedep.be_lowrank(spec, psi0, dt, opts)
    kw = dict(basis_precision=basis) if basis == "dw" else {}
    with gpu_handle(spec) as h:
        phi, psi, st = h.be_step(dt, _dev(psi0), mode="lr", sweep_precision="fp64", dsa_tol=1e-12, **kw, **opts)
    assert st["converged"] == 1 and ref["converged"]
    assert st["outer_iters"] == ref["iters"]
    assert st["total_inner"] == sum(ref["inner"])
    assert rel_l2(phi.cpu().numpy(), ref["phi"]) < 1e-10
    assert rel_l2(_host(psi, d).ravel(), ref["psi"].ravel()) < 1e-9


def test_lowrank_step_fp32_sweeps_and_two_steps_against_full_rank():
    """Mixed precision (FP32 sweeps without the defect correction, double-word basis, FP32 DSA)
    at the paper's tolerances (eps_SI 1e-6, eps_res = eps_diff = 1e-7; FP32 sweeps alone cannot
    reach much below): two low-rank steps track the FP64 full-rank steps of the same problem."""
    spec = _spec(40, 36, seed=23, ratio_range=(0.5, 0.95))
    d = oracle_disc(spec)
    psi0 = _twin_symmetric(d, _psi0(d, 24))
    dt = 0.5
    with gpu_handle(spec) as h:
        psi_l, psi_f = _dev(psi0), _dev(psi0)
        for k in range(2):
            phi_f, psi_f, st_f = h.be_step(dt, psi_f, mode="fr", sweep_precision="fp64", eps_si=1e-11,
                                           dsa_tol=1e-10, max_outer=300)
            phi_l, psi_l, st_l = h.be_step(dt, psi_l, mode="lr", sweep_precision="fp32", sweep_refine=0,
                                           basis_precision="dw", dsa_precision="fp32", dsa_tol=1e-6, eps_si=1e-6,
                                           eps_res=1e-7, eps_diff=1e-7, eps_svd=1e-8, p=4, q=16, seed=5,
                                           max_outer=300)
            assert st_f["converged"] == 1 and st_l["converged"] == 1
            assert rel_l2(phi_l.cpu().numpy(), phi_f.cpu().numpy()) < 1e-4
            assert rel_l2(psi_l.cpu().numpy(), psi_f.cpu().numpy()) < 1e-3


def test_lowrank_step_rejects_asymmetric_previous_flux_and_unsupported_options():
    from paper_2603_25233_gb300._lib import RteError
    spec = _spec(8, 6, seed=25)
    d = oracle_disc(spec)
    with gpu_handle(spec) as h:
        with pytest.raises(RteError, match="twin"):
            h.be_step(0.2, _dev(_psi0(d, 26)), mode="lr", sweep_precision="fp64")
        sym = _dev(_twin_symmetric(d, _psi0(d, 27)))
        for kw in (dict(sampling="deim"), dict(basis_update="qr"), dict(sweep_precision="fp32", sweep_refine=1)):
            with pytest.raises(RteError):
                h.be_step(0.2, sym, mode="lr", **kw)
