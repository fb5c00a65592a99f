"""Diffusion synthetic acceleration correction, Eq. (DSA) / Eq. (diffusion-correction).

Oracle (test infrastructure only).  The paper takes a "fully consistent" discretisation
defined in another work and solves it with AMG-preconditioned CG (Sec. 4); its matrices
are not given.  Reading used here and by the CUDA library: the modified interior-penalty
(MIP) symmetric DG discretisation of

    -div( D grad dphi ) + sigma_a dphi = sigma_s (phi^{(n,*)} - phi^{(n-1)}),   D = 1/(3 sigma_t)

on the same Q1 space, with
    interior faces:  kappa [[u]][[v]] - {{D d_n u}}[[v]] - [[u]]{{D d_n v}},
                     kappa = max(1/4, (C/2)(D^-/h^- + D^+/h^+)),
    boundary faces:  kappa u v - 1/2 (D d_n u) v - 1/2 u (D d_n v),  kappa = max(1/4, C D/h),
with C = 8 = 4 p (p+1) for p = 1 and h the cell width normal to the face.  The matrix is
SPD, so CG applies.  D = 1/(3 sigma_t) replaces the 1/sigma_s of Eq. (diffusion-correction)
(undefined in pure absorbers); sum_j omega_j Omega_x^2 = 1/3 for the CL rule.  The
correction only changes iteration counts: the SI-DSA fixed point is the S_N solution.
Every integral below is computed by Gauss quadrature.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

C_IP = 8.0


def _trace_data(disc):
    b = disc.basis
    ys, wy = b.vface_quad()
    xs, wx = b.hface_quad()
    faces = {}
    # (values, normal derivative in +axis direction) at each cell edge
    v, dx, _ = b.eval(np.full_like(ys, disc.hx / 2), ys)
    faces['R'] = (v, dx, wy)
    v, dx, _ = b.eval(np.full_like(ys, -disc.hx / 2), ys)
    faces['L'] = (v, dx, wy)
    v, _, dy = b.eval(xs, np.full_like(xs, disc.hy / 2))
    faces['T'] = (v, dy, wx)
    v, _, dy = b.eval(xs, np.full_like(xs, -disc.hy / 2))
    faces['B'] = (v, dy, wx)
    return faces


def mip_matrix(disc):
    """Assemble the MIP diffusion matrix (SPD) for the correction equation."""
    N = disc.ndof
    D = 1.0 / (3.0 * disc.sig_t)
    sig_a = disc.sig_t - disc.sig_s
    b = disc.basis
    X, Y, W = b.cell_quad()
    v, dx, dy = b.eval(X, Y)
    stiff = (dx * W) @ dx.T + (dy * W) @ dy.T
    mass = (v * W) @ v.T
    rows, cols, vals = [], [], []

    def add(ci, cj, blk):
        for k in range(4):
            for l in range(4):
                rows.append(4 * ci + k)
                cols.append(4 * cj + l)
                vals.append(blk[k, l])

    for c in range(disc.nc):
        add(c, c, D[c] * stiff + sig_a[c] * mass)
    tr = _trace_data(disc)

    def interior(cm, cp, side_m, side_p, h):
        # face between cell cm ("-" side, normal points from cm to cp) and cp ("+" side)
        vm, dm, w = tr[side_m]
        vp, dp, _ = tr[side_p]
        kap = max(0.25, 0.5 * C_IP * (D[cm] / h + D[cp] / h))
        jumps = {cm: vm, cp: -vp}
        avgs = {cm: 0.5 * D[cm] * dm, cp: 0.5 * D[cp] * dp}
        for A in (cm, cp):
            for B in (cm, cp):
                blk = (kap * (jumps[A] * w) @ jumps[B].T
                       - (jumps[A] * w) @ avgs[B].T
                       - (avgs[A] * w) @ jumps[B].T)
                add(A, B, blk)

    def boundary(c, side, sign, h):
        # sign = +1 if the outward normal is the +axis direction, -1 otherwise
        vv, dd, w = tr[side]
        kap = max(0.25, C_IP * D[c] / h)
        dn = sign * D[c] * dd
        blk = kap * (vv * w) @ vv.T - 0.5 * (vv * w) @ dn.T - 0.5 * (dn * w) @ vv.T
        add(c, c, blk)

    nx, ny = disc.nx, disc.ny
    for iy in range(ny):
        for ix in range(nx):
            c = iy * nx + ix
            if ix + 1 < nx:
                interior(c, c + 1, 'R', 'L', disc.hx)
            if iy + 1 < ny:
                interior(c, c + nx, 'T', 'B', disc.hy)
            if ix == 0:
                boundary(c, 'L', -1.0, disc.hx)
            if ix == nx - 1:
                boundary(c, 'R', +1.0, disc.hx)
            if iy == 0:
                boundary(c, 'B', -1.0, disc.hy)
            if iy == ny - 1:
                boundary(c, 'T', +1.0, disc.hy)
    return sp.csc_matrix((vals, (rows, cols)), shape=(N, N))


class MIPSolver:
    """Direct sparse solve of the MIP correction system (the exact linear-system solution
    that the paper's CG reaches to its relative tolerance)."""

    def __init__(self, disc):
        self.disc = disc
        self.A = mip_matrix(disc)
        self.lu = spla.splu(self.A)

    def correction(self, phi_star, phi_prev):
        """delta phi solving A_MIP dphi = Sigma_s (phi^{(n,*)} - phi^{(n-1)}) (Eq. DSA, reading)."""
        return self.lu.solve(self.disc.Ss @ (phi_star - phi_prev))
