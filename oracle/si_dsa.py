"""Full-rank SI-DSA, Sec. 2.2 (Eq. SI, Eq. DSA) with the loop and stopping rule of Alg. 1.

Oracle (test infrastructure only).  One iteration:
  1. phi^{(n,*)} = sum_j omega_j psi_j,  (D_j + Sigma_t) psi_j = Sigma_s phi^{(n-1)} + G~_j   (Eq. SI)
  2. stop if || phi^{(n,*)} - phi^{(n-1)} ||_inf <= eps_SI                                     (Alg. 1)
  3. phi^{(n)} = phi^{(n,*)} + delta phi  with the DSA correction                              (Eq. DSA)
Readings: the stop test is taken before the DSA step, as Alg. 1 writes it; on exit the
returned flux is phi^{(n,*)}; the loop runs over n <= N_iter; phi^{(0)} = 0 (Sec. 4).

Also provides the direct solve of the coupled S_N system (Eq. mat-vec-a) that pins the
fixed point independently of the iteration and of the DSA discretisation.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .transport import DirectSweeper
from .dsa import MIPSolver


def fr_si_dsa(disc, eps_si=1e-8, max_iter=100, use_dsa=True, phi0=None,
              sweeper=None, mip=None):
    sweeper = sweeper or DirectSweeper(disc)
    mip = mip or (MIPSolver(disc) if use_dsa else None)
    phi = np.zeros(disc.ndof) if phi0 is None else np.array(phi0, dtype=np.float64)
    diffs = []
    converged = False
    n = 0
    for n in range(1, max_iter + 1):
        S = disc.scattering_source(phi)
        phi_star = sweeper.scalar_flux(S)
        diff = np.max(np.abs(phi_star - phi))
        diffs.append(diff)
        if diff <= eps_si:
            phi = phi_star
            converged = True
            break
        phi = phi_star + (mip.correction(phi_star, phi) if use_dsa else 0.0)
    return dict(phi=phi, iters=n, diffs=diffs, converged=converged)


def si_step(disc, phi_prev, sweeper=None, angles=None):
    """One full-rank SI step phi^{(n,*)} from phi^{(n-1)} (Eq. SI)."""
    sweeper = sweeper or DirectSweeper(disc)
    return sweeper.scalar_flux(disc.scattering_source(phi_prev), angles)


def coupled_direct_solve(disc):
    """Solve the whole S_N system of Eq. (mat-vec-a) at once:
       (D_j + Sigma_t) psi_j - Sigma_s sum_k omega_k psi_k = G + g_j^bc  for every j,
    as one sparse LU over all N_x * N_Omega unknowns (tiny grids only).  Returns phi, psi."""
    N, M = disc.ndof, disc.n_angles
    blocks = []
    for j in range(M):
        row = []
        for k in range(M):
            B = -disc.w[k] * disc.Ss
            if k == j:
                B = B + disc.L(j)
            row.append(B)
        blocks.append(row)
    A = sp.bmat(blocks, format='csc')
    rhs = np.concatenate([disc.G + disc.gbc(j) for j in range(M)])
    psi = spla.splu(A).solve(rhs).reshape(M, N).T
    return psi @ disc.w, psi
