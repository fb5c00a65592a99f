"""Discrete adjoint of the S_N system and gradients of a linear detector response.

Oracle (test infrastructure only).  The paper has no adjoint; this is the plain
discrete adjoint of Eq. (mat-vec-a).  For the response R = d^T phi with
(D_j + Sigma_t) psi_j = Sigma_s phi + G + g_j^bc and phi = sum_j omega_j psi_j, the
Lagrangian gives the adjoint system
    (D_j + Sigma_t)^T mu_j = d + Sigma_s chi,   chi = sum_j omega_j mu_j,
and, for per-cell constant sigma_t, sigma_s and source q (orthonormal basis, mass = I):
    dR/dsigma_t,c = - sum_j omega_j mu_j|_c . psi_j|_c
    dR/dsigma_s,c =   chi|_c . phi|_c
    dR/dq_c       =   chi|_c . (int_cell eta_m)_m
The adjoint scalar flux chi is obtained by SI-DSA on the transposed system (same MIP
correction, which is symmetric).
"""
import numpy as np

from .transport import DirectSweeper
from .dsa import MIPSolver


def adjoint_scalar_flux(disc, d, eps_si=1e-13, max_iter=500, sweeper=None, mip=None):
    sweeper = sweeper or DirectSweeper(disc)
    mip = mip or MIPSolver(disc)
    chi = np.zeros(disc.ndof)
    for n in range(1, max_iter + 1):
        src = d + disc.Ss @ chi
        chi_star = np.zeros(disc.ndof)
        for j in range(disc.n_angles):
            chi_star += disc.w[j] * sweeper.solve_transpose(j, src)
        diff = np.max(np.abs(chi_star - chi))
        if diff <= eps_si:
            return chi_star, n
        chi = chi_star + mip.correction(chi_star, chi)
    return chi, max_iter


def gradients(disc, phi, d, chi=None, sweeper=None, mip=None, eps_si=1e-13):
    """Return dict(sig_t=[nc], sig_s=[nc], q=[nc], chi=...) for R = d^T phi at the converged phi."""
    sweeper = sweeper or DirectSweeper(disc)
    if chi is None:
        chi, _ = adjoint_scalar_flux(disc, d, eps_si=eps_si, sweeper=sweeper, mip=mip)
    S = disc.scattering_source(phi)
    asrc = d + disc.Ss @ chi
    g_t = np.zeros(disc.nc)
    for j in range(disc.n_angles):
        psi = sweeper.sweep(j, S)
        mu = sweeper.solve_transpose(j, asrc)
        g_t -= disc.w[j] * (mu * psi).reshape(disc.nc, 4).sum(axis=1)
    g_s = (chi * phi).reshape(disc.nc, 4).sum(axis=1)
    g_q = chi.reshape(disc.nc, 4) @ disc.cell_int
    return dict(sig_t=g_t, sig_s=g_s, q=g_q, chi=chi)
