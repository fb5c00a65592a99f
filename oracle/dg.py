"""Upwind DG-Q1 discretisation of the S_N system, Sec. 2.1 and App. B.

Oracle (test infrastructure only).  Everything here is computed from the integral
definitions with Gauss quadrature on each cell and face:

* the orthonormal local basis eta_k of Q^1 on a cell is obtained by Gram-Schmidt of the
  monomials {1, x, y, xy} (local coordinates) in the cell L2 inner product (Sec. 2.1,
  "orthonormal basis");
* D_x^+-, D_y^+- follow the App. B definitions (Eq. mat-def): volume term
  -int d_x eta_k eta_l plus, over every vertical face, -int (eta_k^+ - eta_k^-) eta_l^+- dy,
  with basis functions extended by zero outside the domain;
* Sigma_t, Sigma_s are int sigma eta_k eta_l; G(k) = int G eta_k; the inflow vector g_j^bc
  is built from int g eta_k over the boundary faces.

Reading of App. B's g^bc (its printed signs contradict the weak form of Sec. 2.1, where
the inflow face term sits on the left-hand side with a minus sign): moved to the
right-hand side it is
   g_j^bc(k) = max(Ox,0) int g(x_L,y) eta_k(x_L^+,y) dy - min(Ox,0) int g(x_R,y) eta_k(x_R^-,y) dy
             + max(Oy,0) int g(x,y_B) eta_k(x,y_B^+) dx - min(Oy,0) int g(x,y_T) eta_k(x,y_T^-) dx.
The constant-solution (infinite medium) test pins this sign.

DOF numbering: global index 4*c + m, cell c = iy*nx + ix, local m = 0..3 for the basis
functions built from 1, x, y, xy (Legendre degrees (0,0), (1,0), (0,1), (1,1)).
"""
import numpy as np
import scipy.sparse as sp

from .quadrature import cl_quadrature

_NG = 3  # Gauss points per direction: exact for the polynomial degrees met here


def _gauss(a, b, n=_NG):
    t, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * t + 0.5 * (a + b), 0.5 * (b - a) * w


class LocalBasis:
    """Orthonormal Q1 basis on the cell [-hx/2, hx/2] x [-hy/2, hy/2] (local coordinates)."""

    def __init__(self, hx, hy):
        self.hx, self.hy = hx, hy
        xs, wx = _gauss(-hx / 2, hx / 2)
        ys, wy = _gauss(-hy / 2, hy / 2)
        X, Y = np.meshgrid(xs, ys)
        W = np.outer(wy, wx)
        mono = np.stack([np.ones_like(X), X, Y, X * Y]).reshape(4, -1)
        W = W.ravel()
        coef = np.zeros((4, 4))
        for m in range(4):
            v = np.zeros(4)
            v[m] = 1.0
            for n in range(m):
                ip = np.sum((v @ mono) * (coef[n] @ mono) * W)
                v = v - ip * coef[n]
            nrm = np.sqrt(np.sum((v @ mono) ** 2 * W))
            coef[m] = v / nrm
        self.coef = coef

    def eval(self, x, y):
        """Values, d/dx and d/dy of the 4 basis functions at local points: arrays [4, npts]."""
        x = np.asarray(x, dtype=np.float64).ravel()
        y = np.asarray(y, dtype=np.float64).ravel()
        one, zero = np.ones_like(x), np.zeros_like(x)
        mono = np.stack([one, x, y, x * y])
        mdx = np.stack([zero, one, zero, y])
        mdy = np.stack([zero, zero, one, x])
        return self.coef @ mono, self.coef @ mdx, self.coef @ mdy

    # -- cell integrals ----------------------------------------------------
    def cell_quad(self):
        xs, wx = _gauss(-self.hx / 2, self.hx / 2)
        ys, wy = _gauss(-self.hy / 2, self.hy / 2)
        X, Y = np.meshgrid(xs, ys)
        return X.ravel(), Y.ravel(), np.outer(wy, wx).ravel()

    def vface_quad(self):
        ys, wy = _gauss(-self.hy / 2, self.hy / 2)
        return ys, wy

    def hface_quad(self):
        xs, wx = _gauss(-self.hx / 2, self.hx / 2)
        return xs, wx


class Discretisation:
    """Assembled S_N upwind DG-Q1 system for one problem (Eq. mat-vec)."""

    def __init__(self, nx, ny, x0, x1, y0, y1, sig_t, sig_s, n_theta, n_omz,
                 q_cell=None, q_rects=(), inflow=(0.0, 0.0, 0.0, 0.0), q_gauss=()):
        self.nx, self.ny = int(nx), int(ny)
        self.x0, self.x1, self.y0, self.y1 = float(x0), float(x1), float(y0), float(y1)
        self.hx = (self.x1 - self.x0) / self.nx
        self.hy = (self.y1 - self.y0) / self.ny
        self.nc = self.nx * self.ny
        self.ndof = 4 * self.nc
        self.sig_t = np.asarray(sig_t, dtype=np.float64).ravel().copy()
        self.sig_s = np.asarray(sig_s, dtype=np.float64).ravel().copy()
        self.q_cell = None if q_cell is None else np.asarray(q_cell, dtype=np.float64).ravel().copy()
        self.q_rects = [tuple(r) for r in q_rects]
        self.q_gauss = [tuple(float(v) for v in g) for g in q_gauss]
        self.inflow = tuple(float(g) for g in inflow)
        self.n_theta, self.n_omz = int(n_theta), int(n_omz)
        self.Ox, self.Oy, self.Oz, self.w = cl_quadrature(self.n_theta, self.n_omz)
        self.n_angles = len(self.w)
        self.basis = LocalBasis(self.hx, self.hy)
        self._assemble()

    @classmethod
    def from_spec(cls, spec, **overrides):
        kw = dict(nx=spec.nx, ny=spec.ny, x0=spec.x0, x1=spec.x1, y0=spec.y0, y1=spec.y1,
                  sig_t=spec.sig_t, sig_s=spec.sig_s, n_theta=spec.n_theta, n_omz=spec.n_omz,
                  q_cell=spec.q_cell, q_rects=spec.q_rects, inflow=spec.inflow,
                  q_gauss=getattr(spec, 'q_gauss', ()))
        kw.update(overrides)
        return cls(**kw)

    # ------------------------------------------------------------------
    def cell_index(self, ix, iy):
        return iy * self.nx + ix

    def _local_matrices(self):
        b = self.basis
        X, Y, W = b.cell_quad()
        v, dx, dy = b.eval(X, Y)
        self.mass = (v * W) @ v.T                  # int eta_k eta_l
        self.vol_x = (dx * W) @ v.T                # int d_x eta_k eta_l   [k, l]
        self.vol_y = (dy * W) @ v.T
        ys, wy = b.vface_quad()
        vR, _, _ = b.eval(np.full_like(ys, self.hx / 2), ys)    # right edge of a cell
        vL, _, _ = b.eval(np.full_like(ys, -self.hx / 2), ys)   # left edge
        self.tRR = (vR * wy) @ vR.T
        self.tLL = (vL * wy) @ vL.T
        self.tLR = (vL * wy) @ vR.T   # test on left edge of the right cell, trial on right edge of the left cell
        self.tRL = (vR * wy) @ vL.T
        self.eL = vL @ wy              # int eta_k(left edge) dy
        self.eR = vR @ wy
        xs, wx = b.hface_quad()
        vT, _, _ = b.eval(xs, np.full_like(xs, self.hy / 2))
        vB, _, _ = b.eval(xs, np.full_like(xs, -self.hy / 2))
        self.tTT = (vT * wx) @ vT.T
        self.tBB = (vB * wx) @ vB.T
        self.tBT = (vB * wx) @ vT.T
        self.tTB = (vT * wx) @ vB.T
        self.eB = vB @ wx
        self.eT = vT @ wx
        self.cell_int = v @ W          # int eta_k over a cell

    def _block_coo(self, rows_c, cols_c, blk, scale=None):
        """COO triplets placing the 4x4 block blk (times a per-entry scale) at cell pairs."""
        rows_c = np.asarray(rows_c)
        cols_c = np.asarray(cols_c)
        R, C, V = [], [], []
        for k in range(4):
            for l in range(4):
                R.append(4 * rows_c + k)
                C.append(4 * cols_c + l)
                val = np.full(rows_c.shape, blk[k, l])
                if scale is not None:
                    val = val * scale
                V.append(val)
        return np.concatenate(R), np.concatenate(C), np.concatenate(V)

    def _assemble(self):
        self._local_matrices()
        nx, ny, N = self.nx, self.ny, self.ndof
        cells = np.arange(self.nc)
        ix = cells % nx
        iy = cells // nx

        def mat(trips):
            R = np.concatenate([t[0] for t in trips])
            C = np.concatenate([t[1] for t in trips])
            V = np.concatenate([t[2] for t in trips])
            return sp.csr_matrix((V, (R, C)), shape=(N, N))

        # --- x faces: left cell Lc = (a-1, b), right cell Rc = (a, b) -------------
        interior_x = ix > 0
        Rc = cells[interior_x]
        Lc = Rc - 1
        last_col = cells[ix == nx - 1]
        first_col = cells[ix == 0]
        vol = self._block_coo(cells, cells, -self.vol_x)
        # D_x^-: trial on the "-" side (left cell of each face)
        self.Dxm = mat([vol,
                        self._block_coo(Lc, Lc, self.tRR),          # test in Lc: +eta_k^- eta_l^-
                        self._block_coo(Rc, Lc, -self.tLR),         # test in Rc: -eta_k^+ eta_l^-
                        self._block_coo(last_col, last_col, self.tRR)])  # right boundary face
        # D_x^+: trial on the "+" side (right cell of each face)
        self.Dxp = mat([vol,
                        self._block_coo(Lc, Rc, self.tRL),          # test in Lc: +eta_k^- eta_l^+
                        self._block_coo(Rc, Rc, -self.tLL),         # test in Rc: -eta_k^+ eta_l^+
                        self._block_coo(first_col, first_col, -self.tLL)])  # left boundary face
        # --- y faces: bottom cell Bc = (a, b-1), top cell Tc = (a, b) -------------
        interior_y = iy > 0
        Tc = cells[interior_y]
        Bc = Tc - nx
        top_row = cells[iy == ny - 1]
        bottom_row = cells[iy == 0]
        voly = self._block_coo(cells, cells, -self.vol_y)
        self.Dym = mat([voly,
                        self._block_coo(Bc, Bc, self.tTT),
                        self._block_coo(Tc, Bc, -self.tBT),
                        self._block_coo(top_row, top_row, self.tTT)])
        self.Dyp = mat([voly,
                        self._block_coo(Bc, Tc, self.tTB),
                        self._block_coo(Tc, Tc, -self.tBB),
                        self._block_coo(bottom_row, bottom_row, -self.tBB)])
        self.St = mat([self._block_coo(cells, cells, self.mass, None)]).multiply(
            np.repeat(self.sig_t, 4)[:, None]).tocsr()
        self.Ss = mat([self._block_coo(cells, cells, self.mass, None)]).multiply(
            np.repeat(self.sig_s, 4)[:, None]).tocsr()
        # boundary vectors: int eta_k over the boundary faces of the boundary cells
        self.e_left = np.zeros(N)
        self.e_right = np.zeros(N)
        self.e_bottom = np.zeros(N)
        self.e_top = np.zeros(N)
        for k in range(4):
            self.e_left[4 * first_col + k] = self.eL[k]
            self.e_right[4 * last_col + k] = self.eR[k]
            self.e_bottom[4 * bottom_row + k] = self.eB[k]
            self.e_top[4 * top_row + k] = self.eT[k]
        self.G = self._source_moments()

    def _source_moments(self):
        """G(k) = int G eta_k (App. B), G = per-cell constants plus rectangle indicators plus
        Gaussians.  Rectangle overlaps are integrated exactly (Gauss quadrature on the overlap)."""
        G = np.zeros(self.ndof)
        if self.q_cell is not None:
            G += (self.q_cell[:, None] * self.cell_int[None, :]).ravel()
        for (rx0, rx1, ry0, ry1, val) in self.q_rects:
            ia0 = max(int(np.floor((rx0 - self.x0) / self.hx)) - 1, 0)
            ia1 = min(int(np.ceil((rx1 - self.x0) / self.hx)) + 1, self.nx)
            ib0 = max(int(np.floor((ry0 - self.y0) / self.hy)) - 1, 0)
            ib1 = min(int(np.ceil((ry1 - self.y0) / self.hy)) + 1, self.ny)
            for ib in range(ib0, ib1):
                cy0 = self.y0 + ib * self.hy
                oy0, oy1 = max(cy0, ry0), min(cy0 + self.hy, ry1)
                if oy1 <= oy0:
                    continue
                for ia in range(ia0, ia1):
                    cx0 = self.x0 + ia * self.hx
                    ox0, ox1 = max(cx0, rx0), min(cx0 + self.hx, rx1)
                    if ox1 <= ox0:
                        continue
                    xs, wx = _gauss(ox0, ox1)
                    ys, wy = _gauss(oy0, oy1)
                    X, Y = np.meshgrid(xs - (cx0 + self.hx / 2), ys - (cy0 + self.hy / 2))
                    v, _, _ = self.basis.eval(X, Y)
                    c = ib * self.nx + ia
                    G[4 * c:4 * c + 4] += val * (v @ np.outer(wy, wx).ravel())
        if self.q_gauss:
            # smooth sources: Gauss-Legendre quadrature of 24 x 24 points per cell
            xs, wx = _gauss(-self.hx / 2, self.hx / 2, 24)
            ys, wy = _gauss(-self.hy / 2, self.hy / 2, 24)
            X, Y = np.meshgrid(xs, ys)
            v, _, _ = self.basis.eval(X, Y)
            vw = v * np.outer(wy, wx).ravel()[None, :]
            for c in range(self.nc):
                xc = self.x0 + (c % self.nx + 0.5) * self.hx
                yc = self.y0 + (c // self.nx + 0.5) * self.hy
                f = np.zeros(X.size)
                for (gx, gy, a, amp) in self.q_gauss:
                    f += amp * np.exp(-a * ((xc + X.ravel() - gx) ** 2 + (yc + Y.ravel() - gy) ** 2))
                G[4 * c:4 * c + 4] += vw @ f
        return G

    def rect_functional(self, rect):
        """Vector d with d . phi = int_rect phi_h (exact overlap integrals), e.g. a detector."""
        saved_q, saved_r, saved_g = self.q_cell, self.q_rects, self.q_gauss
        self.q_cell, self.q_rects, self.q_gauss = None, [tuple(rect) + (1.0,)], []
        d = self._source_moments()
        self.q_cell, self.q_rects, self.q_gauss = saved_q, saved_r, saved_g
        return d

    # ------------------------------------------------------------------
    def D(self, j):
        """Upwind streaming operator D_j, Eq. (upwind-operator)."""
        ox, oy = self.Ox[j], self.Oy[j]
        Dx = self.Dxm if ox >= 0 else self.Dxp
        Dy = self.Dym if oy >= 0 else self.Dyp
        return ox * Dx + oy * Dy

    def L(self, j):
        """D_j + Sigma_t (the operator a transport sweep inverts)."""
        return (self.D(j) + self.St).tocsc()

    def gbc(self, j, inflow=None):
        """Inflow vector g_j^bc for isotropic constant inflow per side (reading in the header)."""
        gL, gR, gB, gT = self.inflow if inflow is None else inflow
        ox, oy = self.Ox[j], self.Oy[j]
        return (max(ox, 0.0) * gL * self.e_left - min(ox, 0.0) * gR * self.e_right
                + max(oy, 0.0) * gB * self.e_bottom - min(oy, 0.0) * gT * self.e_top)

    def gbc_function(self, ox, oy, gfun):
        """Inflow vector for a space-dependent inflow gfun(side, s) (side in 'LRBT', s the
        coordinate along the side), same reading as gbc()."""
        N = self.ndof
        out = np.zeros(N)
        ys, wy = self.basis.vface_quad()
        xs, wx = self.basis.hface_quad()
        if ox > 0:
            vL, _, _ = self.basis.eval(np.full_like(ys, -self.hx / 2), ys)
            for iy in range(self.ny):
                yc = self.y0 + (iy + 0.5) * self.hy
                c = iy * self.nx
                out[4 * c:4 * c + 4] += ox * (vL @ (wy * gfun('L', yc + ys)))
        if ox < 0:
            vR, _, _ = self.basis.eval(np.full_like(ys, self.hx / 2), ys)
            for iy in range(self.ny):
                yc = self.y0 + (iy + 0.5) * self.hy
                c = iy * self.nx + self.nx - 1
                out[4 * c:4 * c + 4] += -ox * (vR @ (wy * gfun('R', yc + ys)))
        if oy > 0:
            vB, _, _ = self.basis.eval(xs, np.full_like(xs, -self.hy / 2))
            for ix in range(self.nx):
                xc = self.x0 + (ix + 0.5) * self.hx
                c = ix
                out[4 * c:4 * c + 4] += oy * (vB @ (wx * gfun('B', xc + xs)))
        if oy < 0:
            vT, _, _ = self.basis.eval(xs, np.full_like(xs, self.hy / 2))
            for ix in range(self.nx):
                xc = self.x0 + (ix + 0.5) * self.hx
                c = (self.ny - 1) * self.nx + ix
                out[4 * c:4 * c + 4] += -oy * (vT @ (wx * gfun('T', xc + xs)))
        return out

    def project_function(self, f):
        """L2 projection coefficients int f eta_k of a function f(x, y) (Gauss quadrature)."""
        X, Y, W = self.basis.cell_quad()
        v, _, _ = self.basis.eval(X, Y)
        out = np.zeros(self.ndof)
        for c in range(self.nc):
            xc = self.x0 + (c % self.nx + 0.5) * self.hx
            yc = self.y0 + (c // self.nx + 0.5) * self.hy
            out[4 * c:4 * c + 4] = v @ (W * f(xc + X, yc + Y))
        return out

    def l2_error(self, coeffs, f, n=5):
        """|| u_h - f ||_L2 over the domain with n x n Gauss points per cell."""
        xs, wx = _gauss(-self.hx / 2, self.hx / 2, n)
        ys, wy = _gauss(-self.hy / 2, self.hy / 2, n)
        X, Y = np.meshgrid(xs, ys)
        W = np.outer(wy, wx).ravel()
        v, _, _ = self.basis.eval(X, Y)
        err2 = 0.0
        for c in range(self.nc):
            xc = self.x0 + (c % self.nx + 0.5) * self.hx
            yc = self.y0 + (c // self.nx + 0.5) * self.hy
            uh = coeffs[4 * c:4 * c + 4] @ v
            err2 += np.sum(W * (uh - f(xc + X.ravel(), yc + Y.ravel())) ** 2)
        return np.sqrt(err2)

    def scattering_source(self, phi):
        """Sigma_s phi + G (right-hand side of Eq. SI without the inflow term)."""
        return self.Ss @ phi + self.G
