"""Backward-Euler time marching of the S_N-DG system, Sec. 3.7.

Oracle (test infrastructure only).  One backward-Euler step of length dt (particle speed 1)
solves the steady system of Eq. (mat-vec-a) with the total cross section modified by the
mass matrix, and the previous step's angular flux as an angle-dependent source:
    (D_j + Sigma_t + M / dt) psi_j^{n+1} - Sigma_s phi^{n+1} = G + g_j^bc + M psi_j^n / dt
for every ordinate j, phi^{n+1} = sum_j omega_j psi_j^{n+1}.

Readings (the paper states the modified cross section Sigma~_t = Sigma_t + M/dt and no more):
  * the time derivative is discretised as (psi^{n+1} - psi^n)/dt, so the source the modified
    cross section implies is M psi^n / dt;
  * M is assembled here from its definition (int eta_k eta_l on every cell); with the
    orthonormal local basis it is the identity, so Sigma_t + M/dt is the mass matrix of
    sigma_t + 1/dt per cell;
  * the SI of a step is Eq. (SI) with the extra source, stopped as in Alg. 1 (max-norm change of
    phi before the DSA step), returning phi^{(n,*)} and the psi of its last sweep;
  * its DSA step is the MIP correction of the modified medium (sigma_t + 1/dt, i.e.
    sigma_a + 1/dt), the diffusion limit of the modified transport operator;
  * warm-started sampling (the combination Sec. 3.6 proposes for implicit time marching: initial
    angular samples from the previous step's angular basis by DEIM, the rank-adaptive loop
    adapting from there): every inner loop of a low-rank step starts from the DEIM points of the
    previous step's right singular vectors V (N_Omega x r', Sec. 3.3's truncation), taken over one
    direction of each +-Omega_z twin pair (the smaller index), r' of them, instead of p random
    angles; the first step of a march, having no previous basis, starts at random.

psi arrays are [N_x, N_Omega] (one column per ordinate), as in si_dsa.coupled_direct_solve.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .dg import Discretisation
from .dsa import MIPSolver


def global_mass(disc):
    """M: block diagonal of the local mass matrix int eta_k eta_l over every cell."""
    return sp.block_diag([sp.csr_matrix(disc.mass)] * disc.nc, format='csc')


def step_operator(disc, j, dt, M=None):
    """D_j + Sigma_t + M / dt."""
    M = global_mass(disc) if M is None else M
    return (disc.L(j) + M / dt).tocsc()


def be_coupled_solve(disc, psi_prev, dt):
    """One step as a single sparse LU over all N_x * N_Omega unknowns (tiny grids only).
    Returns phi^{n+1}, psi^{n+1}."""
    N, Mn = disc.ndof, disc.n_angles
    M = global_mass(disc)
    blocks = []
    for j in range(Mn):
        row = []
        for k in range(Mn):
            B = -disc.w[k] * disc.Ss
            if k == j:
                B = B + step_operator(disc, j, dt, M)
            row.append(B)
        blocks.append(row)
    A = sp.bmat(blocks, format='csc')
    rhs = np.concatenate([disc.G + disc.gbc(j) + M @ psi_prev[:, j] / dt for j in range(Mn)])
    psi = spla.splu(A).solve(rhs).reshape(Mn, N).T
    return psi @ disc.w, psi


class _StepSweeper:
    """psi_j = (D_j + Sigma_t + M/dt)^{-1} rhs by sparse LU, cached per (Omega_x, Omega_y)."""

    def __init__(self, disc, dt):
        self.disc, self.dt = disc, dt
        self.M = global_mass(disc)
        self._lu = {}

    def solve(self, j, rhs):
        key = (self.disc.Ox[j], self.disc.Oy[j])
        lu = self._lu.get(key)
        if lu is None:
            lu = spla.splu(step_operator(self.disc, j, self.dt, self.M))
            self._lu[key] = lu
        return lu.solve(np.asarray(rhs, dtype=np.float64))


def be_si_dsa(spec, psi_prev, dt, eps_si=1e-10, max_iter=500, use_dsa=True, phi0=None):
    """One step by SI-DSA: sweep every ordinate with source Sigma_s phi + G + g_j + M psi_j^n/dt,
    stop on the max-norm change of phi, DSA with the MIP operator of sigma_t + 1/dt.
    Returns dict(phi, psi, iters, converged)."""
    disc = Discretisation.from_spec(spec)
    mod = Discretisation.from_spec(spec, sig_t=np.asarray(spec.sig_t, dtype=np.float64) + 1.0 / dt)
    mip = MIPSolver(mod) if use_dsa else None
    sw = _StepSweeper(disc, dt)
    extra = [sw.M @ psi_prev[:, j] / dt for j in range(disc.n_angles)]
    phi = np.zeros(disc.ndof) if phi0 is None else np.array(phi0, dtype=np.float64)
    psi = np.zeros((disc.ndof, disc.n_angles))
    converged = False
    n = 0
    for n in range(1, max_iter + 1):
        S = disc.scattering_source(phi)
        for j in range(disc.n_angles):
            psi[:, j] = sw.solve(j, S + disc.gbc(j) + extra[j])
        phi_star = psi @ disc.w
        if np.max(np.abs(phi_star - phi)) <= eps_si:
            phi = phi_star
            converged = True
            break
        phi = phi_star + (mip.correction(phi_star, phi) if use_dsa else 0.0)
    return dict(phi=phi, psi=psi.copy(), iters=n, converged=converged)


def be_march(spec, psi0, dt, n_steps):
    """n_steps backward-Euler steps from psi0 by the coupled solve; returns the list of
    (phi, psi) after each step."""
    disc = Discretisation.from_spec(spec)
    out = []
    psi = np.array(psi0, dtype=np.float64)
    for _ in range(n_steps):
        phi, psi = be_coupled_solve(disc, psi, dt)
        out.append((phi, psi))
    return out


def warm_start_angles(disc, V):
    """The initial samples of a warm-started step: the DEIM points of the columns of V (the
    previous step's right singular vectors, N_Omega x r') among one direction of each +-Omega_z
    twin pair (the smaller index), min(r', distinct directions) of them."""
    from . import lowrank
    twin = lowrank.twin_map(disc)
    allowed = [j for j in range(disc.n_angles) if j <= twin[j]]
    return lowrank.deim_points(np.asarray(V, dtype=np.float64), allowed, np.asarray(V).shape[1])


def be_lowrank(spec, psi_prev, dt, opts=None, trace=None, warm_V=None):
    """One step by the low-rank SI-DSA of Alg. 1 applied to the step's steady problem: the
    medium of sigma_t + 1/dt (D_j + Sigma_t + M/dt with M the identity, as pinned) and the
    angle-dependent source psi_j^n / dt in every ordinate's right-hand side (sampled sweeps,
    Galerkin systems, residuals, full check).  psi^{n+1} = X C, the low-rank angular flux of the
    last inner loop.  psi_prev must be equal on +-Omega_z twins (the low-rank SI solves a twin
    pair once).  warm_V: the previous step's V; every inner loop then starts from its DEIM points
    (warm_start_angles).  Returns dict(phi, psi, iters, inner, ranks, converged, V, init_angles),
    V = the right singular vectors of this step's last truncation."""
    from . import lowrank
    disc = Discretisation.from_spec(spec)
    M = global_mass(disc)
    extra = np.column_stack([M @ psi_prev[:, j] / dt for j in range(disc.n_angles)])
    twin = lowrank.twin_map(disc)
    for j in range(disc.n_angles):
        if not np.array_equal(psi_prev[:, j], psi_prev[:, twin[j]]):
            raise ValueError("psi_prev differs on a +-Omega_z twin pair")
    mod = Discretisation.from_spec(spec, sig_t=np.asarray(spec.sig_t, dtype=np.float64) + 1.0 / dt)
    o = dict(opts or {})
    init = None
    if warm_V is not None:
        init = warm_start_angles(disc, warm_V)
        o['init_angles'] = init
    r = lowrank.lowrank_si_dsa(mod, o, trace=trace, extra=extra)
    last = r['last']
    return dict(phi=r['phi'], psi=last['X'] @ last['C'], iters=r['iters'], inner=r['inner'], ranks=r['ranks'],
                converged=r['converged'], V=last.get('V'), init_angles=init)


def be_march_lowrank(spec, psi0, dt, n_steps, opts=None, warm=True):
    """n_steps low-rank backward-Euler steps from psi0 (equal on +-Omega_z twins); with warm,
    each step after the first starts its inner loops from the previous step's basis
    (be_lowrank's warm_V).  Returns the list of be_lowrank results."""
    out = []
    psi = np.array(psi0, dtype=np.float64)
    V = None
    for _ in range(n_steps):
        r = be_lowrank(spec, psi, dt, opts, warm_V=V if warm else None)
        out.append(r)
        psi = r['psi']
        V = r['V']
    return out
