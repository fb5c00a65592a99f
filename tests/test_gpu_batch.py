"""GPU parity of the batched entry points (rte_sweep_batch, rte_si_dsa_solve_batch): problems of
uneven mesh size and ordinate count in one launch against the oracle's direct per-ordinate
solves (Sec. 2.2), its coupled direct solve and its SI step, and against the one-problem calls;
low-rank batches (concurrent solves of uneven rank) against the oracle's low-rank SI-DSA and the
one-problem solves."""
import numpy as np
import pytest

import workloads as W
from tests.helpers import gpu_handle, oracle_disc, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1

# uneven meshes: ragged bands, a single band, fewer columns than a band, one cell wide,
# and quadratures of different sizes
BATCH = [((40, 33), 8, 2), ((70, 65), 16, 2), ((5, 4), 8, 2), ((36, 100), 4, 2), ((1, 3), 4, 1),
         ((33, 64), 8, 4)]


def _specs(seed=0):
    return [W.random_small(nx, ny, n_theta=nt, n_omz=nz, seed=seed + i, inflow=(0.3, 0.1, 0.2, 0.4),
                           box=(0.0, 1.3, -0.2, 0.9))
            for i, ((nx, ny), nt, nz) in enumerate(BATCH)]


def _api():
    from paper_2603_25233_gb300 import api
    return api


def test_sweep_batch_fp64_matches_direct_solves():
    from oracle.transport import DirectSweeper
    api = _api()
    specs = _specs(1)
    hs = [gpu_handle(s) for s in specs]
    try:
        rng = np.random.default_rng(5)
        angles, srcs, S = [], [], []
        for h in hs:
            a = rng.permutation(h.n_angles)[: max(1, h.n_angles // 2)]
            angles.append(a)
            x = rng.standard_normal(h.n_dof)
            S.append(x)
            srcs.append(torch.tensor(x, device="cuda"))
        psis = api.sweep_batch(hs, angles, srcs, FP64)
        for spec, a, x, psi in zip(specs, angles, S, psis):
            d = oracle_disc(spec)
            sw = DirectSweeper(d)
            P = psi.cpu().numpy().reshape(len(a), d.ndof)
            for k, j in enumerate(a):
                assert rel_l2(P[k], sw.sweep(int(j), x)) < 1e-12, (spec.nx, spec.ny, j)
    finally:
        for h in hs:
            h.close()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_sweep_batch_equals_single_problem_sweeps(prec):
    api = _api()
    specs = _specs(2) + [W.random_small(2, 520, n_theta=4, n_omz=1, seed=9)]   # > 16 bands: one by one
    dt = torch.float32 if prec == FP32 else torch.float64
    tol = 1e-6 if prec == FP32 else 1e-13
    for subset in (specs[:-1], specs):
        hs = [gpu_handle(s) for s in subset]
        try:
            angles = [np.arange(h.n_angles)[::-1].copy() for h in hs]
            srcs = [torch.rand(h.n_dof, dtype=dt, device="cuda") for h in hs]
            psis = api.sweep_batch(hs, angles, srcs, prec, add_inflow=True)
            for h, a, s, p in zip(hs, angles, srcs, psis):
                ref = torch.empty_like(p)
                h.sweep(a, s, prec, psi_out=ref)
                assert rel_l2(p.double().cpu().numpy(), ref.double().cpu().numpy()) < tol
        finally:
            for h in hs:
                h.close()


def test_sweep_batch_rejects_bad_arguments():
    api = _api()
    from paper_2603_25233_gb300._lib import RteError
    specs = _specs(3)[:2]
    hs = [gpu_handle(s) for s in specs]
    try:
        srcs = [torch.zeros(h.n_dof, dtype=torch.float64, device="cuda") for h in hs]
        with pytest.raises(RteError):
            api.sweep_batch(hs, [[0], [hs[1].n_angles]], srcs, FP64)       # angle out of range
        with pytest.raises(RteError):
            big = torch.zeros(2 * hs[0].n_dof + 1, dtype=torch.float64, device="cuda")
            api.sweep_batch(hs, [[0], [0]], [big[1:1 + hs[0].n_dof], srcs[1]], FP64)   # misaligned
    finally:
        for h in hs:
            h.close()


def test_solve_batch_fp64_matches_coupled_direct_solve_and_single_solves():
    from oracle import si_dsa
    api = _api()
    specs = [W.random_small(nx, ny, n_theta=nt, n_omz=nz, seed=20 + i, inflow=(0.2, 0.0, 0.1, 0.3))
             for i, ((nx, ny), nt, nz) in enumerate([((6, 5), 8, 2), ((8, 7), 4, 2), ((3, 8), 8, 1), ((7, 2), 4, 4)])]
    hs = [gpu_handle(s) for s in specs]
    try:
        opts = dict(mode="fr", sweep_precision="fp64", eps_si=1e-12, max_outer=500)
        phis, stats = api.si_dsa_solve_batch(hs, **opts)
        for spec, h, phi, st in zip(specs, hs, phis, stats):
            assert st["converged"] == 1
            phi_c, _ = si_dsa.coupled_direct_solve(oracle_disc(spec))
            assert rel_l2(phi.cpu().numpy(), phi_c) < 1e-10
            phi1, st1 = h.si_dsa_solve(**opts)
            assert st1["outer_iters"] == st["outer_iters"]
            assert rel_l2(phi.cpu().numpy(), phi1.cpu().numpy()) < 1e-13
    finally:
        for h in hs:
            h.close()


def test_solve_batch_problems_stop_independently():
    api = _api()
    # a pure absorber converges in two outer iterations; a diffusive problem takes many more
    easy = W.random_small(40, 40, n_theta=8, n_omz=2, seed=30, ratio_range=(0.0, 0.0))
    hard = W.random_small(50, 45, n_theta=8, n_omz=2, seed=31, ratio_range=(0.95, 0.99))
    hs = [gpu_handle(easy), gpu_handle(hard)]
    try:
        phis, stats = api.si_dsa_solve_batch(hs, mode="fr", sweep_precision="fp64", eps_si=1e-10)
        assert all(s["converged"] for s in stats)
        assert stats[0]["outer_iters"] <= 2 < stats[1]["outer_iters"]
        for h, p, s in zip(hs, phis, stats):
            p1, s1 = h.si_dsa_solve(mode="fr", sweep_precision="fp64", eps_si=1e-10)
            assert s1["outer_iters"] == s["outer_iters"]
            assert rel_l2(p.cpu().numpy(), p1.cpu().numpy()) < 1e-12
    finally:
        for h in hs:
            h.close()


def test_solve_batch_with_a_large_problem_uses_the_cooperative_cg():
    """A batch holding a mesh above the cluster-resident CG size (520 x 510 cells) runs the
    cooperative multi-block CG with per-problem reductions; it must equal the one-problem
    solves."""
    api = _api()
    specs = [W.random_small(520, 510, n_theta=4, n_omz=1, seed=40, ratio_range=(0.5, 0.95)),
             W.random_small(40, 37, n_theta=8, n_omz=2, seed=41, ratio_range=(0.9, 0.99))]
    hs = [gpu_handle(s) for s in specs]
    try:
        phis, stats = api.si_dsa_solve_batch(hs, mode="fr", sweep_precision="fp64", eps_si=1e-10)
        for h, p, s in zip(hs, phis, stats):
            assert s["converged"] == 1
            p1, s1 = h.si_dsa_solve(mode="fr", sweep_precision="fp64", eps_si=1e-10)
            assert s1["outer_iters"] == s["outer_iters"]
            assert rel_l2(p.cpu().numpy(), p1.cpu().numpy()) < 1e-11
    finally:
        for h in hs:
            h.close()


def test_solve_batch_rejects_duplicates():
    api = _api()
    from paper_2603_25233_gb300._lib import RteError
    h = gpu_handle(W.random_small(6, 6, seed=1))
    try:
        for mode in ("fr", "lr"):
            with pytest.raises(RteError):
                api.si_dsa_solve_batch([h, h], mode=mode)
    finally:
        h.close()


# low-rank batches: uneven meshes and quadratures (hence uneven ranks), solved concurrently
LR_BATCH = [((8, 6), 16, 2), ((10, 9), 8, 2), ((6, 6), 16, 4), ((12, 5), 8, 2), ((5, 11), 16, 2)]


def test_lowrank_batch_fp64_matches_oracle():
    """Every problem of a low-rank batch (Alg. 1, FP64 sweeps and basis) reproduces the oracle's
    low-rank SI-DSA: outer and inner counts and phi within 1e-10."""
    from oracle import lowrank
    api = _api()
    specs = [W.random_small(nx, ny, n_theta=nt, n_omz=nz, seed=50 + i, inflow=(0.2, 0.1, 0.0, 0.3))
             for i, ((nx, ny), nt, nz) in enumerate(LR_BATCH)]
    opts = dict(eps_si=1e-9, eps_res=1e-10, eps_diff=1e-10, p=1, q=4, seed=11)
    hs = [gpu_handle(s) for s in specs]
    try:
        phis, stats = api.si_dsa_solve_batch(hs, mode="lr", sweep_precision="fp64", **opts)
        for spec, phi, st in zip(specs, phis, stats):
            ref = lowrank.lowrank_si_dsa(oracle_disc(spec), opts)
            assert st["converged"] == 1 and ref["converged"]
            assert st["outer_iters"] == ref["iters"]
            assert st["total_inner"] == sum(ref["inner"])
            assert rel_l2(phi.cpu().numpy(), ref["phi"]) < 1e-10
    finally:
        for h in hs:
            h.close()


@pytest.mark.parametrize("basis", ["fp64", "dw"])
def test_lowrank_batch_of_uneven_ranks_equals_single_solves(basis):
    """The homogeneous Gaussian-source problems of Sec. 4.1 at L = 2, 3 (32^2 and 48^2 cells,
    128 and 288 ordinates) with sigma_s = 0.1, 1, 10, 100: eight problems of uneven size and
    rank (ranks below N_Omega / 2) at the paper's tolerances, mixed precision (FP32 sweeps with
    the FP64 defect correction, FP32 DSA), p = 8 of q = 32.  The concurrent batch gives each
    problem the statistics and phi of its own rte_si_dsa_solve on the same handle (whose CG
    schedule is tuned by then)."""
    api = _api()
    specs = [W.homogeneous_gaussian_e1(L, s) for L in (2, 3) for s in (0.1, 1.0, 10.0, 100.0)]
    opts = dict(mode="lr", sweep_precision="fp32", sweep_refine=1, dsa_precision="fp32", dsa_tol=1e-8,
                eps_si=1e-6, eps_res=1e-7, eps_diff=1e-7, eps_svd=1e-8, p=8, q=32, seed=5, max_outer=300,
                basis_precision=basis)
    hs = [gpu_handle(s) for s in specs]
    try:
        single = [h.si_dsa_solve(**opts) for h in hs]
        phis, stats = api.si_dsa_solve_batch(hs, **opts)
        assert len({s["max_rank"] for s in stats}) > 3          # uneven ranks, some below the cap
        assert any(s["max_rank"] < h.n_angles // 2 for s, h in zip(stats, hs))
        for (p1, s1), p, s in zip(single, phis, stats):
            assert s["converged"] == 1 and s1["converged"] == 1
            for key in ("outer_iters", "total_inner", "max_rank", "final_rank", "breakdowns", "mgs_failures"):
                assert s[key] == s1[key], key
            assert rel_l2(p.cpu().numpy(), p1.cpu().numpy()) < 1e-13
    finally:
        for h in hs:
            h.close()


def test_lowrank_batch_reports_a_failing_problem_and_recovers():
    """A zero Galerkin pivot injected on the host into one problem of a low-rank batch: the call
    returns RTE_ERR_SINGULAR (raised with the problem's index), the other problems still finish,
    and the next batch call on the same handles reproduces the single solves."""
    api = _api()
    from paper_2603_25233_gb300 import _lib as L
    from paper_2603_25233_gb300._lib import RteError
    specs = [W.random_small(16, 16, n_theta=16, n_omz=2, seed=70 + i) for i in range(3)]
    opts = dict(mode="lr", sweep_precision="fp64", eps_si=1e-9, eps_res=1e-10, eps_diff=1e-10, p=2, q=8, seed=3)
    hs = [gpu_handle(s) for s in specs]
    try:
        single = [h.si_dsa_solve(**opts) for h in hs]
        hs[1].inject_failure(L.RTE_ERR_SINGULAR)
        with pytest.raises(RteError, match="problem 1"):
            api.si_dsa_solve_batch(hs, **opts)
        phis, stats = api.si_dsa_solve_batch(hs, **opts)
        for (p1, s1), p, s in zip(single, phis, stats):
            assert s["converged"] == 1 and s["total_inner"] == s1["total_inner"]
            assert rel_l2(p.cpu().numpy(), p1.cpu().numpy()) < 1e-13
    finally:
        for h in hs:
            h.close()


def test_c4_batch_mixed_precision_fixed_point_against_oracle():
    """The 64-problem uneven batch (64^2..256^2 cells, 128..512 ordinates) in one batched
    solve with FP32 sweeps, FP64 defect correction and FP32 DSA.  Every problem must be a fixed
    point of the FP64 SI map evaluated by FP64 GPU sweeps, and the smallest problem's must also
    agree with the oracle's SI step (all its ordinates by sparse LU)."""
    from oracle import si_dsa
    api = _api()
    specs = W.batched_c4()
    hs = [gpu_handle(s) for s in specs]
    try:
        # the stop test is absolute (max-norm change of phi); these fluxes peak near 1e-4, so
        # 1e-11 is a relative change of ~1e-7
        phis, stats = api.si_dsa_solve_batch(hs, mode="fr", sweep_precision="fp32", dsa_precision="fp32",
                                             sweep_refine=1, eps_si=1e-11, max_outer=400)
        assert all(s["converged"] for s in stats), [s["outer_iters"] for s in stats]
        for spec, h, phi in zip(specs, hs, phis):
            G = h.source()
            sig_s = torch.tensor(np.repeat(spec.sig_s, 4), device="cuda")
            S = sig_s * phi + G
            nxt = torch.empty_like(phi)
            h.sweep(np.arange(h.n_angles), S, FP64, phi_out=nxt)
            assert rel_l2(nxt.cpu().numpy(), phi.cpu().numpy()) < 1e-5
        k = min(range(len(specs)), key=lambda i: specs[i].nx * specs[i].ny * specs[i].n_theta * specs[i].n_omz)
        d = oracle_disc(specs[k])
        phi_k = phis[k].cpu().numpy()
        assert rel_l2(si_dsa.si_step(d, phi_k), phi_k) < 1e-5
    finally:
        for h in hs:
            h.close()
