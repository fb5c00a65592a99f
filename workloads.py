"""Seeded synthetic problem descriptions for the steady 2D x-y S_N transport problem.

This module only describes physical inputs: the mesh, per-cell cross sections,
the isotropic source (per-cell constants, axis-aligned rectangles and Gaussians), the
isotropic inflow per domain side and the CL(N_theta, N_Omega_z) quadrature
orders.  It holds none of the discretisation or solver arithmetic: both the
oracle and the CUDA library compute moments, operators and sweeps from these
arrays on their own.  Every random input is drawn from a seeded numpy
generator.

Cell ordering: cell c = iy * nx + ix (row-major, x fastest); cell centre
(x0 + (ix + 1/2) hx, y0 + (iy + 1/2) hy).  Piecewise-constant materials take
the value of the defining field at the cell centre.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np


@dataclass
class ProblemSpec:
    nx: int
    ny: int
    x0: float
    x1: float
    y0: float
    y1: float
    n_theta: int
    n_omz: int
    sig_t: np.ndarray                      # [nx*ny] float64
    sig_s: np.ndarray                      # [nx*ny] float64
    q_cell: Optional[np.ndarray] = None    # [nx*ny] float64 per-cell constant source, or None
    q_rects: List[Tuple[float, float, float, float, float]] = field(default_factory=list)
    inflow: Tuple[float, float, float, float] = (0.0, 0.0, 0.0, 0.0)  # left, right, bottom, top
    name: str = ""
    # isotropic Gaussian sources (xc, yc, a, amp): amp * exp(-a ((x - xc)^2 + (y - yc)^2))
    q_gauss: List[Tuple[float, float, float, float]] = field(default_factory=list)

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny

    @property
    def n_dof(self) -> int:
        return 4 * self.nx * self.ny

    @property
    def n_angles(self) -> int:
        return self.n_theta * self.n_omz

    def cell_centres(self):
        hx = (self.x1 - self.x0) / self.nx
        hy = (self.y1 - self.y0) / self.ny
        xc = self.x0 + (np.arange(self.nx) + 0.5) * hx
        yc = self.y0 + (np.arange(self.ny) + 0.5) * hy
        X, Y = np.meshgrid(xc, yc)          # [ny, nx]
        return X.ravel(), Y.ravel()


def _spec(nx, ny, box, n_theta, n_omz, sig_t, sig_s, q_cell=None, q_rects=(), inflow=(0, 0, 0, 0), name="",
          q_gauss=()):
    return ProblemSpec(nx, ny, float(box[0]), float(box[1]), float(box[2]), float(box[3]),
                       int(n_theta), int(n_omz),
                       np.ascontiguousarray(sig_t, dtype=np.float64),
                       np.ascontiguousarray(sig_s, dtype=np.float64),
                       None if q_cell is None else np.ascontiguousarray(q_cell, dtype=np.float64),
                       [tuple(float(v) for v in r) for r in q_rects], tuple(float(g) for g in inflow), name,
                       [tuple(float(v) for v in g) for g in q_gauss])


# ---------------------------------------------------------------------------
# Configurations with the shapes of the paper's benchmark problems
# ---------------------------------------------------------------------------

def homogeneous_c1(nx: int = 32, ny: int = 32, n_theta: int = 16, n_omz: int = 4) -> ProblemSpec:
    """Unit square, constant sigma_t=1, sigma_s=0.9, q=1 everywhere, vacuum inflow."""
    n = nx * ny
    return _spec(nx, ny, (0, 1, 0, 1), n_theta, n_omz, np.ones(n), np.full(n, 0.9),
                 q_cell=np.ones(n), name=f"homogeneous {nx}x{ny} CL({n_theta},{n_omz})")


def multiscale_c2(nx: int = 128, ny: int = 128, n_theta: int = 32, n_omz: int = 8,
                  eps_left: float = 1e-3) -> ProblemSpec:
    """Two-region multiscale medium on [0,1]^2: sigma_t = 1/eps, sigma_s = 1/eps - eps with
    eps = eps_left on x < 0.5 and eps = 1 on x >= 0.5; q = 1 on [0.4,0.6]^2; vacuum inflow."""
    X, _ = _spec(nx, ny, (0, 1, 0, 1), 1, 1, np.ones(nx * ny), np.ones(nx * ny)).cell_centres()
    eps = np.where(X < 0.5, eps_left, 1.0)
    return _spec(nx, ny, (0, 1, 0, 1), n_theta, n_omz, 1.0 / eps, 1.0 / eps - eps,
                 q_rects=[(0.4, 0.6, 0.4, 0.6, 1.0)],
                 name=f"multiscale {nx}x{ny} CL({n_theta},{n_omz})")


def checkerboard_c3(cells_per_block: int = 64, n_theta: int = 64, n_omz: int = 8) -> ProblemSpec:
    """7x7 checkerboard lattice on [0,7]^2: block (i,j) is an absorber (sigma_t=10, sigma_s=0)
    when i+j is odd, else background (sigma_t=sigma_s=1); q=1 in the centre block (3,3)."""
    nb = 7
    n = nb * cells_per_block
    spec = _spec(n, n, (0, 7, 0, 7), n_theta, n_omz, np.ones(n * n), np.ones(n * n))
    X, Y = spec.cell_centres()
    bi = np.floor(X).astype(int)
    bj = np.floor(Y).astype(int)
    absorber = ((bi + bj) % 2) == 1
    sig_t = np.where(absorber, 10.0, 1.0)
    sig_s = np.where(absorber, 0.0, 1.0)
    return _spec(n, n, (0, 7, 0, 7), n_theta, n_omz, sig_t, sig_s,
                 q_rects=[(3.0, 4.0, 3.0, 4.0, 1.0)], name=f"checkerboard {n}x{n} CL({n_theta},{n_omz})")


GAUSS_SOURCE = (0.0, 0.0, 100.0, 1.0)     # exp(-100 (x^2 + y^2)), Sec. 4.1, 4.3, 4.4


def homogeneous_gaussian_e1(L: int, sigma_s: float, n: Optional[int] = None) -> ProblemSpec:
    """Homogeneous medium of Sec. 4.1: [-1,1]^2, no absorption (sigma_t = sigma_s), Gaussian
    source exp(-100 (x^2 + y^2)), zero inflow, a 16L x 16L mesh with the CL(8L, 4L) quadrature
    (n overrides the mesh side, for small parity cases)."""
    n = 16 * L if n is None else n
    nc = n * n
    return _spec(n, n, (-1, 1, -1, 1), 8 * L, 4 * L, np.full(nc, float(sigma_s)), np.full(nc, float(sigma_s)),
                 q_gauss=[GAUSS_SOURCE], name=f"homogeneous sigma_s={sigma_s:g} {n}x{n} CL({8 * L},{4 * L})")


def variable_scattering_e4(n: int = 80, n_theta: int = 40, n_omz: int = 20) -> ProblemSpec:
    """Multiscale variable scattering of Sec. 4.3: [-1,1]^2, no absorption, Gaussian source,
    vacuum; sigma_s = 99.9 r^4 (r^2 - 2)^2 + 0.1 for r <= 1, else 100 (cell-centre values)."""
    spec = _spec(n, n, (-1, 1, -1, 1), 1, 1, np.ones(n * n), np.ones(n * n))
    X, Y = spec.cell_centres()
    r = np.sqrt(X ** 2 + Y ** 2)
    sig = np.where(r <= 1.0, 99.9 * r ** 4 * (r ** 2 - 2.0) ** 2 + 0.1, 100.0)
    return _spec(n, n, (-1, 1, -1, 1), n_theta, n_omz, sig, sig.copy(), q_gauss=[GAUSS_SOURCE],
                 name=f"variable scattering {n}x{n} CL({n_theta},{n_omz})")


def pin_cell_e5(n: int = 80, n_theta: int = 32, n_omz: int = 16) -> ProblemSpec:
    """Pin cell of Sec. 4.4: [-1,1]^2, no absorption, Gaussian source, vacuum;
    sigma_s = 0.1 on |x|, |y| <= 0.5, else 100 (cell-centre values; the interface lies on
    cell edges when n is a multiple of 4)."""
    spec = _spec(n, n, (-1, 1, -1, 1), 1, 1, np.ones(n * n), np.ones(n * n))
    X, Y = spec.cell_centres()
    sig = np.where((np.abs(X) <= 0.5) & (np.abs(Y) <= 0.5), 0.1, 100.0)
    return _spec(n, n, (-1, 1, -1, 1), n_theta, n_omz, sig, sig.copy(), q_gauss=[GAUSS_SOURCE],
                 name=f"pin cell {n}x{n} CL({n_theta},{n_omz})")


# seeds of the eight repeated pin-cell solves (Sec. 4.4 draws them from the system time)
PIN_CELL_SEEDS = tuple(20260140 + i for i in range(8))


def gaussian_random_field(nx: int, ny: int, corr_len: float, seed: int,
                          box=(0.0, 1.0, 0.0, 1.0)) -> np.ndarray:
    """Zero-mean, unit-variance Gaussian random field with covariance exp(-d^2/(2 l^2)) at the
    cell centres, by FFT spectral synthesis on a periodic grid of twice the mesh size."""
    rng = np.random.default_rng(seed)
    hx = (box[1] - box[0]) / nx
    hy = (box[3] - box[2]) / ny
    mx, my = 2 * nx, 2 * ny
    kx = 2 * np.pi * np.fft.fftfreq(mx, d=hx)
    ky = 2 * np.pi * np.fft.fftfreq(my, d=hy)
    KX, KY = np.meshgrid(kx, ky)
    # spectral density of the squared-exponential covariance
    spec = np.exp(-0.5 * corr_len ** 2 * (KX ** 2 + KY ** 2))
    noise = rng.standard_normal((my, mx)) + 1j * rng.standard_normal((my, mx))
    field_ = np.fft.ifft2(np.sqrt(spec) * noise).real[:ny, :nx]
    field_ = (field_ - field_.mean()) / field_.std()
    return field_.ravel()


def grf_adjoint_c5(n: int = 256, n_theta: int = 64, n_omz: int = 8, seed: int = 20260105,
                   scattering_ratio: float = 0.99) -> ProblemSpec:
    """[0,1]^2 with a log-normal sigma_t field (correlation length 0.1), sigma_s = c sigma_t,
    q = 1 on [0,0.1]^2, vacuum inflow."""
    sig_t = np.exp(gaussian_random_field(n, n, 0.1, seed))
    return _spec(n, n, (0, 1, 0, 1), n_theta, n_omz, sig_t, scattering_ratio * sig_t,
                 q_rects=[(0.0, 0.1, 0.0, 0.1, 1.0)], name=f"grf {n}x{n} CL({n_theta},{n_omz})")


DETECTOR_C5 = (0.9, 1.0, 0.9, 1.0)


def batched_c4(n_problems: int = 64, seed: int = 20260104):
    """Independent problems with uneven sizes: side 16*U{4..16} cells, CL(32,4)/CL(32,8)/CL(64,8),
    log-normal sigma_t (correlation length 0.1), scattering ratio U[0.5,0.999], q=1 on a random
    square of side U[0.1,0.3] inside [0,1]^2, vacuum inflow."""
    rng = np.random.default_rng(seed)
    quads = [(32, 4), (32, 8), (64, 8)]
    out = []
    for i in range(n_problems):
        n = 16 * int(rng.integers(4, 17))
        nt, nz = quads[int(rng.integers(0, 3))]
        c = float(rng.uniform(0.5, 0.999))
        side = float(rng.uniform(0.1, 0.3))
        px = float(rng.uniform(0.0, 1.0 - side))
        py = float(rng.uniform(0.0, 1.0 - side))
        sig_t = np.exp(gaussian_random_field(n, n, 0.1, seed * 1000 + i))
        out.append(_spec(n, n, (0, 1, 0, 1), nt, nz, sig_t, c * sig_t,
                         q_rects=[(px, px + side, py, py + side, 1.0)],
                         name=f"batch[{i}] {n}x{n} CL({nt},{nz}) c={c:.3f}"))
    return out


def random_small(nx: int, ny: int, n_theta: int = 8, n_omz: int = 2, seed: int = 0,
                 inflow=(0.0, 0.0, 0.0, 0.0), box=(0.0, 1.0, 0.0, 1.0),
                 sig_range=(0.5, 5.0), ratio_range=(0.0, 0.95)) -> ProblemSpec:
    """Small heterogeneous problem with independent random per-cell materials and source,
    plus one source rectangle not aligned to cell edges (ragged tests)."""
    rng = np.random.default_rng(seed)
    n = nx * ny
    sig_t = rng.uniform(*sig_range, size=n)
    sig_s = sig_t * rng.uniform(*ratio_range, size=n)
    q = rng.uniform(0.0, 2.0, size=n)
    w, h = box[1] - box[0], box[3] - box[2]
    rect = (box[0] + 0.23 * w, box[0] + 0.61 * w, box[2] + 0.17 * h, box[2] + 0.77 * h, 1.5)
    return _spec(nx, ny, box, n_theta, n_omz, sig_t, sig_s, q_cell=q, q_rects=[rect],
                 inflow=inflow, name=f"random {nx}x{ny} CL({n_theta},{n_omz}) seed {seed}")


def infinite_medium(nx: int, ny: int, sig_t: float, sig_s: float, q: float,
                    n_theta: int = 8, n_omz: int = 2, box=(0.0, 1.0, 0.0, 1.0)) -> ProblemSpec:
    """Constant medium with isotropic inflow q/sigma_a on every side: the exact transport
    solution is the constant psi = q/sigma_a for every direction."""
    n = nx * ny
    g = q / (sig_t - sig_s)
    return _spec(nx, ny, box, n_theta, n_omz, np.full(n, sig_t), np.full(n, sig_s),
                 q_cell=np.full(n, q), inflow=(g, g, g, g), name="infinite medium")


def random_unit_directions(n_dirs: int, dim: int, seed: int) -> np.ndarray:
    """Unit-normalised standard normal directions (rows), for directional derivative checks."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n_dirs, dim))
    return v / np.linalg.norm(v, axis=1, keepdims=True)
