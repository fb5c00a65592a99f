"""GPU parity of the sweep, the DSA operator, full-rank SI-DSA and the adjoint gradient
against the FP64 oracle (all calls go through the C ABI via the binding)."""
import numpy as np
import pytest

import workloads as W
from tests.helpers import gpu_handle, oracle_disc, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1

# sizes chosen to span several bands / a ragged tail / fewer columns than a band / 1 cell
SHAPES = [(5, 4), (7, 37), (40, 33), (70, 65), (1, 3), (3, 1), (33, 64)]


def _spec(nx, ny, seed=0, inflow=(0.3, 0.1, 0.2, 0.4), nt=8, nz=2):
    return W.random_small(nx, ny, n_theta=nt, n_omz=nz, seed=seed, inflow=inflow, box=(0.0, 1.3, -0.2, 0.9))


@pytest.mark.parametrize("shape", SHAPES)
def test_quadrature_and_source_moments_match_oracle(shape):
    spec = _spec(*shape)
    d = oracle_disc(spec)
    with gpu_handle(spec) as h:
        ox, oy, oz, w = h.quadrature()
        assert np.abs(ox - d.Ox).max() < 1e-14 and np.abs(oy - d.Oy).max() < 1e-14
        assert np.abs(oz - d.Oz).max() < 1e-14 and np.abs(w - d.w).max() < 1e-15
        G = h.source().cpu().numpy()
        assert np.abs(G - d.G).max() <= 1e-13 * max(1, np.abs(d.G).max())


@pytest.mark.parametrize("chunk", [None, 4])
@pytest.mark.parametrize("shape", SHAPES)
def test_sweep_fp64_matches_direct_solve(shape, chunk):
    """All ordinates in one call or in calls of 4 ordinates (different CTA counts and staging
    reuse): every psi_j equals the direct solve of its upwind system."""
    spec = _spec(*shape, seed=1)
    d = oracle_disc(spec)
    from oracle.transport import DirectSweeper
    sw = DirectSweeper(d)
    rng = np.random.default_rng(2)
    S = rng.standard_normal(d.ndof)
    angles = np.arange(d.n_angles)
    with gpu_handle(spec) as h:
        src = torch.tensor(S, device="cuda")
        psi = torch.empty(len(angles) * d.ndof, dtype=torch.float64, device="cuda")
        phi = torch.empty(d.ndof, dtype=torch.float64, device="cuda")
        if chunk is None:
            h.sweep(angles, src, FP64, psi_out=psi, phi_out=phi)
        else:
            phi.zero_()
            part = torch.empty(d.ndof, dtype=torch.float64, device="cuda")
            for a0 in range(0, len(angles), chunk):
                sub = angles[a0:a0 + chunk]
                h.sweep(sub, src, FP64, psi_out=psi[a0 * d.ndof:(a0 + len(sub)) * d.ndof], phi_out=part)
                phi += part
        P = psi.cpu().numpy().reshape(len(angles), d.ndof)
        ref_phi = np.zeros(d.ndof)
        for a, j in enumerate(angles):
            ref = sw.sweep(j, S)
            assert rel_l2(P[a], ref) < 1e-12, (shape, j)
            ref_phi += d.w[j] * ref
        assert rel_l2(phi.cpu().numpy(), ref_phi) < 1e-12


def test_sweep_per_angle_source_and_no_inflow():
    spec = _spec(9, 11, seed=3)
    d = oracle_disc(spec)
    from oracle.transport import DirectSweeper
    sw = DirectSweeper(d)
    rng = np.random.default_rng(4)
    angles = np.array([3, 0, 15, 7])
    S = rng.standard_normal((len(angles), d.ndof))
    with gpu_handle(spec) as h:
        psi = torch.empty(len(angles) * d.ndof, dtype=torch.float64, device="cuda")
        h.sweep(angles, torch.tensor(S.ravel(), device="cuda"), FP64, src_per_angle=True, add_inflow=False, psi_out=psi)
        P = psi.cpu().numpy().reshape(len(angles), d.ndof)
    for a, j in enumerate(angles):
        assert rel_l2(P[a], sw.solve(j, S[a])) < 1e-12


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_sweep_scrambled_list_per_angle_source_and_repeats(prec):
    """37 ordinates in a scrambled order of all quadrants, a per-ordinate source, a repeated
    ordinate, a ragged 29 x 19 mesh and a non-unit box; then the same list with the shared
    source."""
    spec = W.random_small(29, 19, n_theta=16, n_omz=4, seed=8, inflow=(0.3, 0.1, 0.2, 0.4), box=(0.0, 1.3, -0.2, 0.9))
    d = oracle_disc(spec)
    from oracle.transport import DirectSweeper
    sw = DirectSweeper(d)
    rng = np.random.default_rng(9)
    angles = rng.permutation(d.n_angles)[:36]
    angles = np.append(angles, angles[5])
    S = rng.standard_normal((len(angles), d.ndof))
    dt = torch.float64 if prec == FP64 else torch.float32
    tol = 1e-12 if prec == FP64 else 2e-5
    with gpu_handle(spec) as h:
        psi = torch.empty(len(angles) * d.ndof, dtype=dt, device="cuda")
        h.sweep(angles, torch.tensor(S.ravel(), dtype=dt, device="cuda"), prec, src_per_angle=True, add_inflow=False,
                psi_out=psi)
        P = psi.double().cpu().numpy().reshape(len(angles), d.ndof)
        for a, j in enumerate(angles):
            assert rel_l2(P[a], sw.solve(j, S[a])) < tol, (a, j)
        h.sweep(angles, torch.tensor(S[0], dtype=dt, device="cuda"), prec, psi_out=psi)
        P = psi.double().cpu().numpy().reshape(len(angles), d.ndof)
    for a, j in enumerate(angles):
        assert rel_l2(P[a], sw.sweep(j, S[0])) < tol, (a, j)


@pytest.mark.parametrize("shape", [(40, 33), (70, 65)])
def test_sweep_fp32_within_single_precision(shape):
    spec = _spec(*shape, seed=5)
    d = oracle_disc(spec)
    from oracle.transport import DirectSweeper
    sw = DirectSweeper(d)
    S = np.abs(np.random.default_rng(6).standard_normal(d.ndof))
    angles = np.arange(d.n_angles)
    with gpu_handle(spec) as h:
        psi = torch.empty(len(angles) * d.ndof, dtype=torch.float32, device="cuda")
        h.sweep(angles, torch.tensor(S, dtype=torch.float32, device="cuda"), FP32, psi_out=psi)
        P = psi.cpu().numpy().astype(np.float64).reshape(len(angles), d.ndof)
    for a, j in enumerate(angles):
        assert rel_l2(P[a], sw.sweep(j, S)) < 2e-5


@pytest.mark.parametrize("shape", [(5, 4), (40, 33)])
def test_adjoint_sweep_is_transposed_solve(shape):
    spec = _spec(*shape, seed=7)
    d = oracle_disc(spec)
    from oracle.transport import DirectSweeper
    sw = DirectSweeper(d)
    S = np.random.default_rng(8).standard_normal(d.ndof)
    angles = np.arange(d.n_angles)
    with gpu_handle(spec) as h:
        mu = torch.empty(len(angles) * d.ndof, dtype=torch.float64, device="cuda")
        h.sweep_adjoint(angles, torch.tensor(S, device="cuda"), FP64, mu_out=mu)
        M = mu.cpu().numpy().reshape(len(angles), d.ndof)
    for a, j in enumerate(angles):
        assert rel_l2(M[a], sw.solve_transpose(j, S)) < 1e-12


@pytest.mark.parametrize("shape", [(5, 4), (13, 9), (40, 33)])
def test_dsa_operator_matches_oracle_mip_matrix(shape):
    from oracle.dsa import mip_matrix
    import scipy.sparse.linalg as spla
    spec = _spec(*shape, seed=9)
    d = oracle_disc(spec)
    A = mip_matrix(d)
    x = np.random.default_rng(10).standard_normal(d.ndof)
    with gpu_handle(spec) as h:
        y = h.dsa_apply(torch.tensor(x, device="cuda")).cpu().numpy()
        assert rel_l2(y, A @ x) < 1e-13
        b = A @ x
        sol, it = h.dsa_solve(torch.tensor(b, device="cuda"), tol=1e-13, max_iter=5000)
        assert it > 0
        assert rel_l2(sol.cpu().numpy(), spla.spsolve(A.tocsc(), b)) < 1e-9


@pytest.mark.parametrize("case", ["multiscale", "ragged", "one-row", "one-cell", "mid"])
def test_dsa_two_level_cg_matches_direct_solve_in_few_iterations(case):
    """The DSA CG with the two-level (block Jacobi + vertex multigrid) preconditioner: the
    solution of the MIP system equals a sparse direct solve, and the iteration count stays
    small where block Jacobi alone needs hundreds (optically thick, diffusive half domain)."""
    import scipy.sparse.linalg as spla
    from oracle.dsa import mip_matrix
    spec = {"multiscale": lambda: W.multiscale_c2(64, 64, 8, 2),
            "ragged": lambda: W.random_small(37, 29, seed=3, ratio_range=(0.9, 0.999)),
            "one-row": lambda: W.random_small(45, 1, seed=4),
            "one-cell": lambda: W.random_small(1, 1, seed=5),
            "mid": lambda: W.random_small(301, 290, seed=6, ratio_range=(0.9, 0.999))}[case]()
    d = oracle_disc(spec)
    A = mip_matrix(d).tocsc()
    rng = np.random.default_rng(7)
    b = rng.standard_normal(d.ndof)
    with gpu_handle(spec) as h:
        sol, it = h.dsa_solve(torch.tensor(b, device="cuda"), tol=1e-12, max_iter=5000)
    assert rel_l2(sol.cpu().numpy(), spla.spsolve(A, b)) < 1e-9
    assert it <= 40, it


def test_dsa_cg_above_the_cluster_size_solves_the_mip_system():
    """A mesh above the cluster-resident CG size (520 x 510 cells, 1.06 M unknowns) takes the
    cooperative multi-block CG with the grid-level V-cycle; its solution must satisfy the MIP
    system (operator checked against the oracle's matrix above) to the CG tolerance."""
    spec = W.random_small(520, 510, n_theta=4, n_omz=1, seed=13, ratio_range=(0.9, 0.999))
    with gpu_handle(spec) as h:
        b = torch.randn(h.n_dof, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
        x, it = h.dsa_solve(b, tol=1e-10, max_iter=5000)
        r = h.dsa_apply(x) - b
        assert 0 < it < 200, it
        assert float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(b)) < 1e-9


@pytest.mark.parametrize("shape", [(6, 5), (33, 17)])
def test_fr_si_dsa_fp64_matches_oracle(shape):
    from oracle import si_dsa
    spec = _spec(*shape, seed=11)
    d = oracle_disc(spec)
    ref = si_dsa.fr_si_dsa(d, eps_si=1e-12, max_iter=300)
    with gpu_handle(spec) as h:
        phi, st = h.si_dsa_solve(mode="fr", sweep_precision="fp64", eps_si=1e-12, max_outer=300)
    assert st["converged"] == 1
    assert st["outer_iters"] == ref["iters"]
    assert rel_l2(phi.cpu().numpy(), ref["phi"]) < 1e-10


def test_fr_si_dsa_reaches_coupled_solution_c1_shape():
    """Homogeneous 32x32 problem with CL(16,4) (the 64-ordinate FP64 configuration)."""
    from oracle import si_dsa
    spec = W.homogeneous_c1()
    d = oracle_disc(spec)
    ref = si_dsa.fr_si_dsa(d, eps_si=1e-8)
    with gpu_handle(spec) as h:
        phi, st = h.si_dsa_solve(mode="fr", sweep_precision="fp64", eps_si=1e-8)
    assert st["converged"] == 1 and st["outer_iters"] == ref["iters"]
    assert rel_l2(phi.cpu().numpy(), ref["phi"]) < 1e-10


def test_fr_fp32_sweep_flux_within_1e5():
    from oracle import si_dsa
    spec = W.multiscale_c2(32, 32, 8, 4)
    d = oracle_disc(spec)
    phi_c = si_dsa.fr_si_dsa(d, eps_si=1e-11, max_iter=400)["phi"]
    with gpu_handle(spec) as h:
        phi, st = h.si_dsa_solve(mode="fr", sweep_precision="fp32", eps_si=1e-8, max_outer=400)
    assert st["converged"] == 1
    assert rel_l2(phi.cpu().numpy(), phi_c) < 1e-5


def test_infinite_medium_on_gpu():
    spec = W.infinite_medium(37, 5, 2.0, 1.5, 1.0)
    with gpu_handle(spec) as h:
        phi, st = h.si_dsa_solve(mode="fr", eps_si=1e-14, max_outer=400)
        hx, hy = 1.0 / 37, 1.0 / 5
    P = phi.cpu().numpy().reshape(-1, 4)
    assert np.abs(P[:, 0] - 2.0 * np.sqrt(hx * hy)).max() < 1e-12
    assert np.abs(P[:, 1:]).max() < 1e-12


def test_adjoint_gradient_matches_oracle():
    from oracle import si_dsa
    from oracle.adjoint import gradients
    spec = W.random_small(7, 6, n_theta=8, n_omz=2, seed=12, ratio_range=(0.3, 0.9))
    d = oracle_disc(spec)
    det = d.rect_functional((0.5, 1.0, 0.4, 1.0))
    phi_ref, _ = si_dsa.coupled_direct_solve(d)
    g_ref = gradients(d, phi_ref, det)
    with gpu_handle(spec) as h:
        phi, st = h.si_dsa_solve(mode="fr", eps_si=1e-14, max_outer=500)
        g = h.adjoint_grad(phi, torch.tensor(det, device="cuda"), eps_si=1e-14, max_outer=500)
    for k in ("sig_t", "sig_s", "q"):
        assert rel_l2(g[k].cpu().numpy(), g_ref[k]) < 1e-9, k
