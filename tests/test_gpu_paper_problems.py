"""GPU runs of the paper's analytic experiments (Sec. 4.1 homogeneous medium, Sec. 4.3 variable
scattering, Sec. 4.4 pin cell): the Gaussian source moments against the oracle, step-by-step
low-rank parity with the oracle on reduced meshes, and at the paper's sizes the low-rank solve
against the full-rank solve of the same problem (Sec. 4: equal outer iteration counts and a
scalar-flux difference below the outer tolerance).  The paper's ranks and speedups are not
pinned (its DSA and random streams differ)."""
import numpy as np
import pytest

import workloads as W
from tests.helpers import gpu_handle, oracle_disc, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# Sec. 4 defaults: eps_SI-SA = 1e-6, eps_res = eps_diff = 1e-7, eps_SVD = 1e-8, p = 1, q = 8
PAPER = dict(eps_si=1e-6, eps_res=1e-7, eps_diff=1e-7, eps_svd=1e-8, p=1, q=8)


@pytest.mark.parametrize("make", [lambda: W.homogeneous_gaussian_e1(1, 10.0, n=7),
                                  lambda: W.homogeneous_gaussian_e1(2, 100.0),
                                  lambda: W.variable_scattering_e4(),
                                  lambda: W.pin_cell_e5()])
def test_gaussian_source_moments_match_oracle(make):
    spec = make()
    d = oracle_disc(spec)
    with gpu_handle(spec) as h:
        G = h.source().cpu().numpy()
    assert np.abs(G - d.G).max() <= 1e-13 * np.abs(d.G).max()


TIGHT = dict(eps_si=1e-9, eps_res=1e-10, eps_diff=1e-10)
SMALL = {   # reduced meshes and quadratures; the pin cell converges slowly under the MIP DSA
    "e1-diffusive": (lambda: W.homogeneous_gaussian_e1(1, 100.0, n=8), TIGHT),
    "e1-transport": (lambda: W.homogeneous_gaussian_e1(1, 0.1, n=8), TIGHT),
    "e4": (lambda: W.variable_scattering_e4(10, 8, 4), TIGHT),
    "e5": (lambda: W.pin_cell_e5(12, 8, 4), dict(eps_si=1e-6, eps_res=1e-8, eps_diff=1e-8)),
}


@pytest.mark.parametrize("basis", ["fp64", "dw"])
@pytest.mark.parametrize("case", sorted(SMALL))
def test_reduced_paper_problem_lowrank_matches_oracle_iteration_by_iteration(case, basis):
    from oracle import lowrank
    make, tol = SMALL[case]
    spec = make()
    d = oracle_disc(spec)
    opts = dict(tol, p=1, q=8, seed=20260141)
    ref = lowrank.lowrank_si_dsa(d, opts)
    with gpu_handle(spec) as h:
        phi, st = h.si_dsa_solve(mode="lr", sweep_precision="fp64", basis_precision=basis, **opts)
    assert st["converged"] == 1 and ref["converged"]
    assert st["outer_iters"] == ref["iters"]
    assert st["total_inner"] == sum(ref["inner"])
    assert st["final_rank"] == ref["ranks"][-1]
    assert rel_l2(phi.cpu().numpy(), ref["phi"]) < 1e-10


FULL = {   # E1 at L = 5: 400 distinct directions, a basis capacity beyond 256 columns
    "e1-L5-sigma100": lambda: W.homogeneous_gaussian_e1(5, 100.0),
    "e1-L3-sigma1": lambda: W.homogeneous_gaussian_e1(3, 1.0),
    "e4": lambda: W.variable_scattering_e4(),
    "e5": lambda: W.pin_cell_e5(),
}


@pytest.mark.parametrize("case", sorted(FULL))
def test_paper_problem_lowrank_against_fullrank_at_the_papers_tolerances(case):
    """Mixed-precision low-rank SI-DSA (FP32 sweeps with defect correction, double-word basis
    passes) and the FP64 full-rank SI-DSA, both stopped by the paper's outer test: the outer
    iteration counts agree (the paper reports one exception of one iteration), the fluxes
    differ by less than eps_SI-SA in the 2-norm, and the rank respects the +-Omega_z ceiling.
    Both stop at the same distance from the converged FP64 full-rank flux (the paper's absolute
    eps_SI-SA = 1e-6, against fluxes of order 1e-4, sets that distance, not the low-rank step)."""
    spec = FULL[case]()
    with gpu_handle(spec) as h:
        ref = torch.zeros(h.n_dof, dtype=torch.float64, device="cuda")
        _, st_ref = h.si_dsa_solve(mode="fr", sweep_precision="fp64", eps_si=1e-12, max_outer=400, dsa_tol=1e-12,
                                   phi=ref)
        fr = torch.zeros_like(ref)
        _, st_fr = h.si_dsa_solve(mode="fr", sweep_precision="fp64", eps_si=PAPER["eps_si"], max_outer=400, phi=fr)
        lr = torch.zeros_like(ref)
        _, st_lr = h.si_dsa_solve(mode="lr", sweep_precision="fp32", basis_precision="dw", max_outer=400,
                                  truncate=2, seed=20260141, phi=lr, **PAPER)
    assert st_ref["converged"] == 1 and st_fr["converged"] == 1 and st_lr["converged"] == 1
    assert abs(st_lr["outer_iters"] - st_fr["outer_iters"]) <= 1
    assert float(torch.linalg.vector_norm(lr - fr)) < PAPER["eps_si"]
    assert st_lr["max_rank"] <= h.n_angles // 2
    e_lr = rel_l2(lr.cpu().numpy(), ref.cpu().numpy())
    e_fr = rel_l2(fr.cpu().numpy(), ref.cpu().numpy())
    assert abs(e_lr - e_fr) <= 0.05 * e_fr + 1e-6
