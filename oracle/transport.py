"""Per-ordinate transport solves, Sec. 2.2 (Eq. SI and the block-triangular structure).

Oracle (test infrastructure only).  A transport sweep computes
psi_j = (D_j + Sigma_t)^{-1} b_j exactly (up to rounding order); the oracle computes the
same quantity by a direct sparse LU solve of the assembled per-ordinate system.  The
block Gauss-Seidel pass in upwind order that the paper describes (Sec. 2.2) is also
written out cell by cell for tiny grids, where it pins the direct solve and checks the
block lower-triangular structure.
"""
import numpy as np
import scipy.sparse.linalg as spla


class DirectSweeper:
    """psi_j = (D_j + Sigma_t)^{-1} rhs by sparse LU, factorisations cached per direction."""

    def __init__(self, disc, cache=True):
        self.disc = disc
        self.cache = cache
        self._lu = {}

    def _factor(self, j):
        key = (self.disc.Ox[j], self.disc.Oy[j])   # +-Omega_z twins share (Omega_x, Omega_y)
        lu = self._lu.get(key)
        if lu is None:
            lu = spla.splu(self.disc.L(j))
            if self.cache:
                self._lu[key] = lu
        return lu

    def solve(self, j, rhs):
        return self._factor(j).solve(np.asarray(rhs, dtype=np.float64))

    def solve_transpose(self, j, rhs):
        """(D_j + Sigma_t)^T mu = rhs (used by the adjoint)."""
        return self._factor(j).solve(np.asarray(rhs, dtype=np.float64), trans='T')

    def sweep(self, j, S):
        """One-ordinate SI solve of Eq. (SI): (D_j + Sigma_t) psi_j = S + g_j^bc."""
        return self.solve(j, S + self.disc.gbc(j))

    def scalar_flux(self, S, angles=None):
        """phi = sum_j omega_j psi_j over the given ordinates (all by default)."""
        d = self.disc
        angles = range(d.n_angles) if angles is None else angles
        phi = np.zeros(d.ndof)
        for j in angles:
            phi += d.w[j] * self.sweep(j, S)
        return phi


def upwind_cell_order(disc, j):
    """Cells ordered along the upwind direction of ordinate j (rows, then columns)."""
    xs = range(disc.nx) if disc.Ox[j] >= 0 else range(disc.nx - 1, -1, -1)
    ys = range(disc.ny) if disc.Oy[j] >= 0 else range(disc.ny - 1, -1, -1)
    return [iy * disc.nx + ix for iy in ys for ix in xs]


def block_gauss_seidel_sweep(disc, j, rhs, check_structure=True):
    """The transport sweep as one block Gauss-Seidel pass in upwind order (Sec. 2.2):
    for each cell in upwind order solve A_cc psi_c = b_c - sum_{n upwind} A_cn psi_n.
    With check_structure, asserts that no cell couples to a cell later in the order
    (the block lower-triangular property)."""
    A = disc.L(j).tocsr()
    order = upwind_cell_order(disc, j)
    pos = np.empty(disc.nc, dtype=int)
    pos[order] = np.arange(disc.nc)
    psi = np.zeros(disc.ndof)
    for c in order:
        rows = slice(4 * c, 4 * c + 4)
        blockrows = A[rows, :].tocoo()
        b = np.array(rhs[rows], dtype=np.float64)
        Acc = np.zeros((4, 4))
        for r, col, v in zip(blockrows.row, blockrows.col, blockrows.data):
            n = col // 4
            if n == c:
                Acc[r, col % 4] += v
            else:
                if check_structure and pos[n] > pos[c] and v != 0.0:
                    raise AssertionError("coupling to a downwind cell")
                b[r] -= v * psi[col]
        psi[rows] = np.linalg.solve(Acc, b)
    return psi
