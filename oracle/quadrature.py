"""Chebyshev-Legendre quadrature CL(N_theta, N_Omega_z), App. A.

Oracle (test infrastructure only).  Tensor product of the normalised N_Omega_z-point
Gauss-Legendre rule in Omega_z on [-1, 1] (weights summing to one) and N_theta
equispaced azimuths theta_j = (2j - 1) pi / N_theta with weight 1 / N_theta.

Angle index convention: j = j2 * N_theta + j1 (j1 azimuth, j2 polar node), zero based.
"""
import numpy as np


def cl_quadrature(n_theta: int, n_omz: int):
    """Return (Ox, Oy, Oz, w), each of length n_theta * n_omz (App. A, Eq. for Omega_j, omega_j)."""
    z, wz = np.polynomial.legendre.leggauss(n_omz)
    wz = wz / 2.0                                   # normalised: sum = 1
    j1 = np.arange(1, n_theta + 1)
    theta = (2.0 * j1 - 1.0) * np.pi / n_theta
    Ox = np.empty(n_theta * n_omz)
    Oy = np.empty_like(Ox)
    Oz = np.empty_like(Ox)
    w = np.empty_like(Ox)
    for j2 in range(n_omz):
        s = np.sqrt(1.0 - z[j2] ** 2)
        sl = slice(j2 * n_theta, (j2 + 1) * n_theta)
        Ox[sl] = np.cos(theta) * s
        Oy[sl] = np.sin(theta) * s
        Oz[sl] = z[j2]
        w[sl] = wz[j2] / n_theta
    return Ox, Oy, Oz, w
