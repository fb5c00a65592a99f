"""GPU parity of the rank-adaptive low-rank SI / SI-DSA against the oracle's step-by-step
implementation of Sec. 3 (same Philox4x32-10 candidate keys, so the same angles are drawn
and selected in FP64)."""
import numpy as np
import pytest

import workloads as W
from tests.helpers import gpu_handle, oracle_disc, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _spec(nx, ny, seed=0, nt=16, nz=2, inflow=(0.0, 0.0, 0.0, 0.0)):
    return W.random_small(nx, ny, n_theta=nt, n_omz=nz, seed=seed, inflow=inflow)


# Basis passes in FP64 or in double-word FP32 (about 48 significant bits, Dot2 sums): the
# double-word passes change the iterates by ~1e-14 relative, far below the phi tolerances used
# here, and no rank or iteration-count decision of these cases lies that close to its threshold.
# "dw-tc": the double-word chain with the first projection of every snapshot block on the
# tensor cores (split TF32); the second, double-word projection removes its error.
BASIS = ["fp64", "dw", "dw-tc"]


def basis_kw(basis):
    if basis == "dw-tc":
        return dict(basis_precision="dw", tc_projection=1)
    return dict(basis_precision=basis)


@pytest.mark.parametrize("basis", BASIS)
@pytest.mark.parametrize("shape,p,q,inflow", [((6, 5), 1, 4, (0, 0, 0, 0)),
                                              ((9, 7), 2, 6, (0.3, 0.0, 0.1, 0.2)),
                                              ((33, 17), 1, 8, (0, 0, 0, 0))])
def test_single_lowrank_si_step_matches_oracle(shape, p, q, inflow, basis):
    from oracle import lowrank
    spec = _spec(*shape, seed=3, inflow=inflow)
    d = oracle_disc(spec)
    opts = dict(eps_res=1e-9, eps_diff=1e-9, p=p, q=q, seed=77)
    trace = []
    ref = lowrank.lowrank_si(d, np.zeros(d.ndof), 1, opts, trace=trace)
    with gpu_handle(spec) as h:
        phi, st = h.si_dsa_solve(mode="lr", sweep_precision="fp64", max_outer=1, use_dsa=0, eps_si=0.0,
                                 truncate=0, **basis_kw(basis), **opts)
    assert st["final_rank"] == ref["rank"]
    assert st["total_inner"] == ref["stats"]["inner"]
    assert st["full_checks"] == ref["stats"]["full_checks"]
    assert rel_l2(phi.cpu().numpy(), ref["phi"]) < 1e-11


@pytest.mark.parametrize("basis", BASIS)
def test_lowrank_si_dsa_matches_oracle_iteration_by_iteration(basis):
    from oracle import lowrank
    spec = _spec(8, 6, seed=5, inflow=(0.2, 0.1, 0.0, 0.3))
    d = oracle_disc(spec)
    opts = dict(eps_si=1e-9, eps_res=1e-10, eps_diff=1e-10, p=1, q=4, seed=11)
    ref = lowrank.lowrank_si_dsa(d, opts)
    with gpu_handle(spec) as h:
        phi, st = h.si_dsa_solve(mode="lr", sweep_precision="fp64", **basis_kw(basis), **opts)
    assert st["converged"] == 1 and ref["converged"]
    assert st["outer_iters"] == ref["iters"]
    assert st["total_inner"] == sum(ref["inner"])
    assert rel_l2(phi.cpu().numpy(), ref["phi"]) < 1e-10


def test_lowrank_fixed_point_equals_full_rank():
    from oracle import si_dsa
    spec = _spec(12, 10, seed=6, nt=16, nz=4)
    d = oracle_disc(spec)
    phi_c, _ = si_dsa.coupled_direct_solve(d)
    with gpu_handle(spec) as h:
        phi, st = h.si_dsa_solve(mode="lr", sweep_precision="fp64", eps_si=1e-10, eps_res=1e-11,
                                 eps_diff=1e-11, p=1, q=8)
    assert st["converged"] == 1
    assert st["max_rank"] <= d.n_angles // 2
    assert rel_l2(phi.cpu().numpy(), phi_c) < 1e-8


@pytest.mark.parametrize("basis", BASIS)
def test_lowrank_factors_reconstruct_scalar_flux(basis):
    spec = _spec(10, 9, seed=8, nt=16, nz=4)
    with gpu_handle(spec) as h:
        phi, st = h.si_dsa_solve(mode="lr", sweep_precision="fp64", eps_si=1e-9, eps_res=1e-10,
                                 eps_diff=1e-10, eps_svd=1e-12, want_factors=1, **basis_kw(basis))
        X, S, V = h.factors()
        _, _, _, w = h.quadrature()
    X = X.cpu().numpy()
    V = V.cpu().numpy()
    S = S.cpu().numpy()
    r = len(S)
    assert st["final_rank_trunc"] == r
    assert np.all(np.diff(S) <= 0)
    assert np.abs(X.T @ X - np.eye(r)).max() < 1e-10
    assert np.abs(V.T @ V - np.eye(r)).max() < 1e-10
    phi_rec = X @ (S * (V.T @ w))
    assert rel_l2(phi_rec, phi.cpu().numpy()) < 1e-9


@pytest.mark.parametrize("basis", BASIS)
def test_mixed_precision_lowrank_multiscale_within_1e5(basis):
    from oracle import si_dsa
    spec = W.multiscale_c2(32, 32, 16, 4)
    d = oracle_disc(spec)
    phi_ref = si_dsa.fr_si_dsa(d, eps_si=1e-11, max_iter=500)["phi"]
    with gpu_handle(spec) as h:
        phi, st = h.si_dsa_solve(mode="lr", sweep_precision="fp32", eps_si=1e-8, eps_res=1e-8,
                                 eps_diff=1e-8, p=1, q=8, max_outer=500, seed=20260101, **basis_kw(basis))
    assert st["converged"] == 1
    assert rel_l2(phi.cpu().numpy(), phi_ref) < 1e-5


@pytest.mark.parametrize("basis", BASIS)
def test_lowrank_step_on_the_checkerboard_lattice_equals_full_rank_step(basis):
    """Full-size lattice (448 x 448 cells, CL(64,8) = 512 ordinates, N_x = 802,816): one
    rank-adaptive SI step from phi = 0 with tight inner tolerances (8 sampled angles per inner
    iteration out of 32 candidates) equals the full-rank SI step over all ordinates, i.e. the
    Galerkin-projected angular flux reproduces Sum_j w_j psi_j (Sec. 3, Eq. SI)."""
    spec = W.checkerboard_c3()
    with gpu_handle(spec) as h:
        phi_lr, st = h.si_dsa_solve(mode="lr", sweep_precision="fp64", max_outer=1, use_dsa=0, eps_si=0.0,
                                    eps_res=1e-10, eps_diff=1e-10, p=8, q=32, truncate=0, seed=20260102,
                                    **basis_kw(basis))
        phi_fr, _ = h.si_dsa_solve(mode="fr", sweep_precision="fp64", max_outer=1, use_dsa=0, eps_si=0.0)
    assert st["total_inner"] >= 1 and st["final_rank"] >= 8
    assert rel_l2(phi_lr.cpu().numpy(), phi_fr.cpu().numpy()) < 1e-7


@pytest.mark.parametrize("basis", ["fp64", "dw"])
def test_lowrank_step_with_more_than_256_directions_matches_oracle(basis):
    """CL(64,10) on a 12 x 10 mesh: 320 distinct directions, so the basis grows past 256 columns.
    The double-word chain then takes its unfused passes (the fused pass keeps at most 256 columns'
    products in registers); the FP64 chain is unchanged."""
    from oracle import lowrank
    spec = W.random_small(12, 10, n_theta=64, n_omz=10, seed=4, inflow=(0.1, 0.0, 0.2, 0.0))
    d = oracle_disc(spec)
    opts = dict(eps_res=1e-9, eps_diff=1e-9, p=2, q=8, seed=91)
    ref = lowrank.lowrank_si(d, np.zeros(d.ndof), 1, opts, trace=[])
    assert ref["rank"] > 256
    with gpu_handle(spec) as h:
        phi, st = h.si_dsa_solve(mode="lr", sweep_precision="fp64", max_outer=1, use_dsa=0, eps_si=0.0,
                                 truncate=0, **basis_kw(basis), **opts)
    assert st["final_rank"] == ref["rank"]
    assert st["total_inner"] == ref["stats"]["inner"]
    assert st["full_checks"] == ref["stats"]["full_checks"]
    assert rel_l2(phi.cpu().numpy(), ref["phi"]) < 1e-11


def test_bench_configuration_reaches_the_target_error():
    """The benchmark's own solve at full size (multiscale 128 x 128, CL(32,8), mixed precision,
    double-word basis passes, p = 8 of q = 32, its tolerances) against the converged FP64 full-rank
    solution (itself parity-tested against the oracle on small meshes): the property the benchmark's
    metric is quoted on, relative L2 error below 1e-5."""
    from paper_2603_25233_gb300.api import default_opts
    spec = W.multiscale_c2()
    with gpu_handle(spec) as h:
        ref = torch.zeros(h.n_dof, dtype=torch.float64, device="cuda")
        _, st_fr = h.si_dsa_solve(default_opts(mode="fr", sweep_precision="fp64", eps_si=1e-11, max_outer=400,
                                               dsa_tol=1e-10), phi=ref)
        phi = torch.zeros(h.n_dof, dtype=torch.float64, device="cuda")
        _, st = h.si_dsa_solve(default_opts(mode="lr", sweep_precision="fp32", sweep_refine=1, eps_si=1e-7,
                                            eps_res=1e-8, eps_diff=1e-8, eps_svd=1e-9, p=8, q=32, max_outer=200,
                                            dsa_tol=1e-6, dsa_precision="fp32", truncate=2, seed=20260101,
                                            basis_precision="dw"), phi=phi)
    assert st_fr["converged"] == 1 and st["converged"] == 1
    assert st["max_rank"] <= h.n_angles // 2
    assert rel_l2(phi.cpu().numpy(), ref.cpu().numpy()) < 1e-5


@pytest.mark.parametrize("basis", BASIS)
@pytest.mark.parametrize("eps_svd", [2e-3, 1e-5])
def test_truncation_matches_oracle_singular_values_and_rank(basis, eps_svd):
    """Truncated SVD C = U S V^T of Sec. 3.3 after one low-rank SI step: the GPU's kept singular
    values and r' equal those of the oracle's truncation of its own C (same draws, same basis),
    and the truncated factors reproduce the same rank-r' angular flux X S V^T.  An optically
    thick, nearly pure scatterer, whose singular values decay, so that r' < r."""
    from oracle import lowrank
    n = 10
    spec = W._spec(n, n, (0, 1, 0, 1), 16, 4, np.full(n * n, 50.0), np.full(n * n, 49.9), q_cell=np.ones(n * n),
                   inflow=(0.2, 0.0, 0.1, 0.0))
    d = oracle_disc(spec)
    opts = dict(eps_res=1e-6, eps_diff=1e-6, p=1, q=6, seed=31, eps_svd=eps_svd)
    ref = lowrank.lowrank_si(d, np.zeros(d.ndof), 1, dict(opts, truncate=True))
    s_all = np.linalg.svd(ref["C"], compute_uv=False)
    tail = 1.0 - np.cumsum(s_all) / s_all.sum()
    rp = ref["rank_trunc"]
    # the rule is not decided within rounding: the tail ratio crosses eps_svd clearly at r'
    assert tail[rp - 1] <= eps_svd / 1.01 and (rp == 1 or tail[rp - 2] >= eps_svd * 1.01)
    assert 1 < rp < ref["rank"]
    with gpu_handle(spec) as h:
        phi, st = h.si_dsa_solve(mode="lr", sweep_precision="fp64", max_outer=1, use_dsa=0, eps_si=0.0,
                                 truncate=1, want_factors=1, **basis_kw(basis), **opts)
        X, S, V = (t.cpu().numpy() for t in h.factors())
    assert st["final_rank"] == ref["rank"] and st["final_rank_trunc"] == rp
    assert len(S) == rp
    assert np.abs(S - ref["S"]).max() <= 1e-10 * ref["S"][0]
    psi_gpu = (X * S) @ V.T
    psi_ref = (ref["U_X"] * ref["S"]) @ ref["V"].T
    assert np.abs(psi_gpu - psi_ref).max() <= 1e-9 * np.abs(psi_ref).max()


@pytest.mark.parametrize("basis", ["fp64", "dw"])
@pytest.mark.parametrize("nt,nz,p", [(16, 4, 1), (32, 4, 2), (64, 4, 3)])
def test_fully_greedy_sampling_matches_oracle(nt, nz, p, basis):
    """Fully greedy sampling (remark in Sec. 3.2): q beyond the number of angles makes every
    unsampled angle a candidate, up to 250 candidates an inner iteration (the FP64 candidate
    vectors then run in several 64-wide launches); with p > 1 the top residuals often belong to a
    +-Omega_z twin pair, and the second twin swept is a breakdown (its flux is already in span X)."""
    from oracle import lowrank
    spec = _spec(8, 6, seed=21, nt=nt, nz=nz, inflow=(0.1, 0.0, 0.0, 0.2))
    d = oracle_disc(spec)
    opts = dict(eps_res=1e-9, eps_diff=1e-9, p=p, q=1000, seed=17)
    ref = lowrank.lowrank_si(d, np.zeros(d.ndof), 1, opts)
    with gpu_handle(spec) as h:
        phi, st = h.si_dsa_solve(mode="lr", sweep_precision="fp64", max_outer=1, use_dsa=0, eps_si=0.0,
                                 truncate=0, **basis_kw(basis), **opts)
    assert st["final_rank"] == ref["rank"]
    assert st["total_inner"] == ref["stats"]["inner"]
    assert st["full_checks"] == ref["stats"]["full_checks"]
    assert rel_l2(phi.cpu().numpy(), ref["phi"]) < 1e-11


def test_checkerboard_lattice_mixed_precision_lowrank_solve_reaches_the_target_error():
    """The lattice configuration as configured (448 x 448 cells, CL(64,8) = 512 ordinates, FP32
    sweeps with FP64 defect correction, double-word basis passes, FP64 truncation; p = 8 of q = 32
    angles per inner iteration, eps_SI 1e-7 with the inner tolerances 0.1 eps_SI) against the
    converged FP64 full-rank solution: relative L2 error below 1e-5, same outer iteration count
    as the FP64 full-rank solve stopped by the same outer test."""
    spec = W.checkerboard_c3()
    with gpu_handle(spec) as h:
        ref = torch.zeros(h.n_dof, dtype=torch.float64, device="cuda")
        _, st_ref = h.si_dsa_solve(mode="fr", sweep_precision="fp64", eps_si=1e-11, max_outer=400, dsa_tol=1e-10,
                                   phi=ref)
        fr = torch.zeros_like(ref)
        _, st_fr = h.si_dsa_solve(mode="fr", sweep_precision="fp64", eps_si=1e-7, max_outer=400, dsa_tol=1e-10,
                                  phi=fr)
        lr = torch.zeros_like(ref)
        _, st_lr = h.si_dsa_solve(mode="lr", sweep_precision="fp32", sweep_refine=1, basis_precision="dw",
                                  eps_si=1e-7, eps_res=1e-8, eps_diff=1e-8, eps_svd=1e-9, p=8, q=32, max_outer=400,
                                  dsa_tol=1e-10, truncate=2, seed=20260102, phi=lr)
    assert st_ref["converged"] == 1 and st_fr["converged"] == 1 and st_lr["converged"] == 1
    assert st_lr["outer_iters"] == st_fr["outer_iters"]
    assert st_lr["max_rank"] <= h.n_angles // 2
    assert rel_l2(lr.cpu().numpy(), ref.cpu().numpy()) < 1e-5


@pytest.mark.parametrize("basis", ["fp64", "dw"])
@pytest.mark.parametrize("shape,nt,nz,p,tol", [((10, 8), 16, 4, 2, 1e-6), ((7, 9), 16, 2, 1, 1e-9),
                                               ((12, 10), 32, 4, 3, 1e-5)])
def test_deim_sampling_matches_oracle(shape, nt, nz, p, tol, basis):
    """DEIM sampling (remark in Sec. 3.2): every inner iteration the Galerkin coefficients of all
    angles, their SVD and the DEIM points of the p leading right singular vectors among the
    unsampled angles; the loop stops on the flux change.  Same picks, ranks and flux as the
    oracle's restatement."""
    from oracle import lowrank
    n = shape[0] * shape[1]
    spec = W._spec(shape[0], shape[1], (0, 1, 0, 1), nt, nz, np.full(n, 50.0), np.full(n, 49.9),
                   q_cell=np.ones(n), inflow=(0.2, 0.0, 0.1, 0.0))
    d = oracle_disc(spec)
    opts = dict(eps_res=tol, eps_diff=tol, p=p, q=8, seed=13, sampling="deim")
    trace = []
    ref = lowrank.lowrank_si(d, np.zeros(d.ndof), 1, opts, trace=trace)
    with gpu_handle(spec) as h:
        phi, st = h.si_dsa_solve(mode="lr", sweep_precision="fp64", max_outer=1, use_dsa=0, eps_si=0.0,
                                 truncate=0, **basis_kw(basis), **opts)
    assert st["final_rank"] == ref["rank"]
    assert st["total_inner"] == ref["stats"]["inner"]
    assert st["full_checks"] == ref["stats"]["full_checks"]
    assert rel_l2(phi.cpu().numpy(), ref["phi"]) < 1e-11


@pytest.mark.parametrize("bu", ["mgsqr", "qr"])
@pytest.mark.parametrize("shape,nt,nz,sig", [((8, 12), 16, 2, (3.0, 2.0)), ((12, 12), 32, 4, (5.0, 4.0))])
def test_basis_update_ablation_matches_oracle(shape, nt, nz, sig, bu):
    """The basis-update ablation of Sec. 4.2 (Table 2): a single projection per snapshot with a
    full QR of the basis (CholeskyQR2 on the GPU, Householder in the oracle) on a failed test
    (MGS-QR, the all-column test) or after every inner iteration (QR), every projected operator
    and Galerkin factor rebuilt after it.  Same ranks, inner iterations and flux as the oracle;
    QR: one full QR per inner iteration.  MGS-QR's count of full QRs decides |X^T psi| <= 1e-10
    after one projection, and single-pass losses cluster near that threshold (the oracle's own
    count differs between BLAS builds), so it matches up to the decisions within a factor of 5
    of the threshold (0 on the first case, 16 on the second)."""
    from oracle import lowrank
    n = shape[0] * shape[1]
    spec = W._spec(shape[0], shape[1], (0, 1, 0, 1), nt, nz, np.full(n, sig[0]), np.full(n, sig[1]),
                   q_cell=np.ones(n), inflow=(0.2, 0.0, 0.1, 0.0))
    d = oracle_disc(spec)
    opts = dict(eps_res=1e-9, eps_diff=1e-9, p=1, q=6, seed=31, mgs_test="max", basis_update=bu)
    ref = lowrank.lowrank_si(d, np.zeros(d.ndof), 1, opts)
    with gpu_handle(spec) as h:
        phi, st = h.si_dsa_solve(mode="lr", sweep_precision="fp64", max_outer=1, use_dsa=0, eps_si=0.0,
                                 truncate=0, basis_precision="fp64", **opts)
    assert st["final_rank"] == ref["rank"]
    assert st["total_inner"] == ref["stats"]["inner"]
    if bu == "qr":
        assert st["full_qr"] == ref["stats"]["full_qr"] == ref["stats"]["inner"]
    else:
        near = 0 if shape == (8, 12) else 16
        assert abs(st["full_qr"] - ref["stats"].get("full_qr", 0)) <= near
        if near == 0:
            assert st["full_qr"] == 0
    assert rel_l2(phi.cpu().numpy(), ref["phi"]) < 1e-11


@pytest.mark.parametrize("basis", ["fp64", "dw"])
def test_incremental_projected_operators_equal_direct_products(basis):
    """The projected operators bordered column by column as the basis grows (Sec. 3.4) equal
    X^T D_x^- X, X^T D_y^- X and X^T Sigma_t X formed directly from the oracle's assembled
    matrices and the GPU's final basis, and X is orthonormal (both to 1e-12)."""
    spec = _spec(12, 9, seed=31, nt=16, nz=2)
    d = oracle_disc(spec)
    with gpu_handle(spec) as h:
        h.si_dsa_solve(mode="lr", sweep_precision="fp64", eps_si=1e-9, eps_res=1e-10, eps_diff=1e-10, p=2, q=8,
                       seed=13, **basis_kw(basis))
        stt = h.lowrank_state()
    X = stt["X"].cpu().numpy()
    r = X.shape[1]
    assert 1 < r <= d.n_angles // 2
    assert np.abs(X.T @ X - np.eye(r)).max() < 1e-12
    for name, A in (("Pxm", d.Dxm), ("Pym", d.Dym), ("T", d.St)):
        direct = X.T @ (A @ X)
        got = stt[name].cpu().numpy()
        assert np.abs(got - direct).max() <= 1e-12 * max(1.0, np.abs(direct).max()), name


def test_lowrank_state_requires_a_lowrank_solve():
    from paper_2603_25233_gb300._lib import RteError
    with gpu_handle(_spec(6, 5, seed=32)) as h:
        with pytest.raises(RteError):
            h.lowrank_state()
        h.si_dsa_solve(mode="fr", sweep_precision="fp64", eps_si=1e-9)
        with pytest.raises(RteError):
            h.lowrank_state()
