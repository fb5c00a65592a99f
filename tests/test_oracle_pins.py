"""Pins of the FP64 CPU oracle against values fixed by the paper and by mathematics.

Each test is chosen so that a plausible mistake in the oracle (dropped term, wrong sign,
transposed block, wrong index) fails at least one of them.  CPU only.
"""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import dsa, lowrank, si_dsa
from oracle.adjoint import adjoint_scalar_flux, gradients
from oracle.dg import Discretisation
from oracle.philox import philox4x32_10, draw_without_replacement
from oracle.quadrature import cl_quadrature
from oracle.transport import DirectSweeper, block_gauss_seidel_sweep

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox (KAT)
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])


def test_draw_is_a_subset_without_replacement():
    cand = list(range(3, 40, 2))
    a = draw_without_replacement(7, 2, 5, cand, 6)
    assert len(set(a)) == 6 and set(a) <= set(cand)
    assert a == draw_without_replacement(7, 2, 5, cand, 6)
    assert a != draw_without_replacement(7, 2, 6, cand, 6)
    from oracle.philox import angle_key
    assert draw_without_replacement(7, 2, 5, cand, 100) == sorted(cand, key=lambda j: (angle_key(7, 2, 5, j), j))


# ---------------------------------------------------------------- quadrature (App. A)
def _sphere_moment(a, b, c):
    """(1/4 pi) int_{S^2} x^a y^b z^c: zero unless all even, else 2 G(al)G(be)G(ga)/G(al+be+ga)/(4 pi)."""
    if a % 2 or b % 2 or c % 2:
        return 0.0
    al, be, ga = (a + 1) / 2, (b + 1) / 2, (c + 1) / 2
    return 2 * math.gamma(al) * math.gamma(be) * math.gamma(ga) / math.gamma(al + be + ga) / (4 * math.pi)


@pytest.mark.parametrize("N", [2, 3, 4])
def test_cl_quadrature_exact_to_degree_2N_minus_1(N):
    """App. A states exactness to degree 2N for CL(2N, N); an N-point Gauss-Legendre rule is
    exact to degree 2N - 1 only, which is what holds (z^{2N} is not integrated exactly)."""
    Ox, Oy, Oz, w = cl_quadrature(2 * N, N)
    assert abs(w.sum() - 1) < 1e-14
    for a in range(2 * N):
        for b in range(2 * N - a):
            for c in range(2 * N - a - b):
                got = np.sum(w * Ox ** a * Oy ** b * Oz ** c)
                assert abs(got - _sphere_moment(a, b, c)) < 1e-13, (a, b, c)
    assert abs(np.sum(w * Oz ** (2 * N)) - _sphere_moment(0, 0, 2 * N)) > 1e-3


def test_cl_quadrature_symmetry_and_second_moments():
    Ox, Oy, Oz, w = cl_quadrature(16, 4)
    pts = {(round(x, 12), round(y, 12), round(z, 12)): ww for x, y, z, ww in zip(Ox, Oy, Oz, w)}
    for x, y, z, ww in zip(Ox, Oy, Oz, w):
        assert abs(pts[(round(-x, 12), round(-y, 12), round(-z, 12))] - ww) < 1e-15
    assert abs(np.sum(w * Ox ** 2) - 1 / 3) < 1e-14
    assert abs(np.sum(w * Oy ** 2) - 1 / 3) < 1e-14
    assert np.all(np.abs(Ox) > 1e-3) and np.all(np.abs(Oy) > 1e-3)   # no ordinate on an axis


# ---------------------------------------------------------------- DG operators (App. B)
def _small(nx=5, ny=4, seed=3, inflow=(0.3, 0.1, 0.2, 0.4)):
    return Discretisation.from_spec(W.random_small(nx, ny, seed=seed, inflow=inflow))


def test_basis_orthonormal_and_integration_by_parts():
    d = _small()
    assert np.abs(d.mass - np.eye(4)).max() < 1e-14
    # int d_x(eta_k eta_l) = trace terms on the right minus left edge
    assert np.abs(d.vol_x + d.vol_x.T - (d.tRR - d.tLL)).max() < 1e-13
    assert np.abs(d.vol_y + d.vol_y.T - (d.tTT - d.tBB)).max() < 1e-13


def test_upwind_operators_transpose_identity():
    """The downwind operator is minus the transpose of the upwind one: D^{+T} = -D^-."""
    d = _small()
    assert abs(d.Dxp.T + d.Dxm).max() < 1e-13
    assert abs(d.Dyp.T + d.Dym).max() < 1e-13


def test_upwind_operator_symmetric_part_is_jump_penalty():
    """psi^T D_j psi = 1/2 sum over faces |Omega.n| int [[psi]]^2 >= 0 (boundary faces included)."""
    d = _small()
    rng = np.random.default_rng(0)
    for j in range(d.n_angles):
        v = rng.standard_normal(d.ndof)
        assert v @ (d.D(j) @ v) > 0


def test_infinite_medium_constant_solution():
    """Isotropic inflow q/sigma_a with constant data: the exact S_N-DG solution is constant."""
    spec = W.infinite_medium(5, 4, 2.0, 1.5, 1.0, n_theta=8, n_omz=2, box=(0.0, 1.3, -0.2, 0.7))
    d = Discretisation.from_spec(spec)
    phi, psi = si_dsa.coupled_direct_solve(d)
    exact = np.zeros(d.ndof)
    exact[0::4] = (1.0 / 0.5) * math.sqrt(d.hx * d.hy)
    assert np.abs(phi - exact).max() < 1e-12
    for j in range(d.n_angles):
        assert np.abs(psi[:, j] - exact).max() < 1e-12
    r = si_dsa.fr_si_dsa(d, eps_si=1e-14, max_iter=300)
    assert np.abs(r['phi'] - exact).max() < 1e-12


def _rate(errs, hs):
    return np.log(errs[-2] / errs[-1]) / np.log(hs[-2] / hs[-1])


def test_pure_absorber_exponential_attenuation_second_order():
    """sigma_s = 0, q = 0, exact psi = exp(-sigma (x - x_L)/Omega_x) fed through the inflow."""
    sig = 1.7
    errs, hs = [], []
    for n in (4, 8, 16):
        spec = W._spec(n, n, (0, 1, 0, 1), 8, 2, np.full(n * n, sig), np.zeros(n * n))
        d = Discretisation.from_spec(spec)
        j = 0
        ox, oy = d.Ox[j], d.Oy[j]
        assert ox > 0 and oy > 0

        def exact(x, y):
            return np.exp(-sig * (x - 0.0) / ox) + 0.0 * y

        g = d.gbc_function(ox, oy, lambda side, s: exact(np.zeros_like(s), s) if side == 'L'
                           else exact(s, np.zeros_like(s)))
        psi = DirectSweeper(d).solve(j, g)
        errs.append(d.l2_error(psi, exact))
        hs.append(1.0 / n)
    assert _rate(errs, hs) > 1.9


def test_manufactured_solution_second_order():
    """Smooth psi_ex with source Omega.grad psi + sigma_t psi for one ordinate."""
    errs, hs = [], []
    for n in (4, 8, 16):
        rng_sig = 1.3
        spec = W._spec(n, n, (0, 1, 0, 1), 8, 2, np.full(n * n, rng_sig), np.zeros(n * n))
        d = Discretisation.from_spec(spec)
        j = 5
        ox, oy = d.Ox[j], d.Oy[j]

        def ex(x, y):
            return 2.0 + np.sin(np.pi * x) * np.cos(2 * y)

        def src(x, y):
            return (ox * np.pi * np.cos(np.pi * x) * np.cos(2 * y)
                    - oy * 2 * np.sin(np.pi * x) * np.sin(2 * y) + rng_sig * ex(x, y))

        def gfun(side, s):
            if side == 'L':
                return ex(np.zeros_like(s), s)
            if side == 'R':
                return ex(np.ones_like(s), s)
            if side == 'B':
                return ex(s, np.zeros_like(s))
            return ex(s, np.ones_like(s))

        rhs = d.project_function(src) + d.gbc_function(ox, oy, gfun)
        psi = DirectSweeper(d).solve(j, rhs)
        errs.append(d.l2_error(psi, ex))
        hs.append(1.0 / n)
    assert _rate(errs, hs) > 1.9


def test_direct_solve_equals_upwind_block_gauss_seidel():
    """Sec. 2.2: the sweep is one block Gauss-Seidel pass; the system is block lower
    triangular in upwind order (checked inside the pass)."""
    d = _small(6, 5)
    sw = DirectSweeper(d)
    S = d.scattering_source(np.random.default_rng(1).standard_normal(d.ndof))
    for j in range(d.n_angles):
        a = sw.sweep(j, S)
        b = block_gauss_seidel_sweep(d, j, S + d.gbc(j))
        assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(a).max())


def test_global_particle_balance():
    """Converged phi*: leakage + absorption = source + inflow (eta = 1 test function)."""
    d = _small(6, 5, inflow=(0.5, 0.0, 1.0, 0.25))
    phi, psi = si_dsa.coupled_direct_solve(d)
    b = d.basis
    ys, wy = b.vface_quad()
    xs, wx = b.hface_quad()
    vR, _, _ = b.eval(np.full_like(ys, d.hx / 2), ys)
    vL, _, _ = b.eval(np.full_like(ys, -d.hx / 2), ys)
    vT, _, _ = b.eval(xs, np.full_like(xs, d.hy / 2))
    vB, _, _ = b.eval(xs, np.full_like(xs, -d.hy / 2))
    gL, gR, gB, gT = d.inflow
    leak = 0.0
    inflow = 0.0
    for j in range(d.n_angles):
        ox, oy, w = d.Ox[j], d.Oy[j], d.w[j]
        P = psi[:, j].reshape(d.nc, 4)
        for iy in range(d.ny):
            cl, cr = iy * d.nx, iy * d.nx + d.nx - 1
            if ox > 0:
                leak += w * ox * np.sum(wy * (P[cr] @ vR))
                inflow += w * ox * gL * d.hy
            else:
                leak += w * -ox * np.sum(wy * (P[cl] @ vL))
                inflow += w * -ox * gR * d.hy
        for ix in range(d.nx):
            cb, ct = ix, (d.ny - 1) * d.nx + ix
            if oy > 0:
                leak += w * oy * np.sum(wx * (P[ct] @ vT))
                inflow += w * oy * gB * d.hx
            else:
                leak += w * -oy * np.sum(wx * (P[cb] @ vB))
                inflow += w * -oy * gT * d.hx
    Pphi = phi.reshape(d.nc, 4)
    absorption = np.sum((d.sig_t - d.sig_s) * (Pphi @ d.cell_int))
    source = np.sum(d.G.reshape(d.nc, 4)[:, 0] * d.cell_int[0])
    assert abs(leak + absorption - source - inflow) < 1e-11 * (source + inflow)


def test_fr_si_dsa_reaches_coupled_direct_solution():
    d = _small(6, 5)
    phi_c, _ = si_dsa.coupled_direct_solve(d)
    r = si_dsa.fr_si_dsa(d, eps_si=1e-13, max_iter=300)
    assert r['converged']
    assert np.linalg.norm(r['phi'] - phi_c) <= 1e-10 * np.linalg.norm(phi_c)
    r0 = si_dsa.fr_si_dsa(d, eps_si=1e-13, max_iter=1000, use_dsa=False)
    assert np.linalg.norm(r0['phi'] - phi_c) <= 1e-10 * np.linalg.norm(phi_c)
    assert r['iters'] < r0['iters']


def test_source_moments_of_unaligned_rectangle():
    """Rectangle source integrals: the cell-average moments sum to value * area and
    the first moments give value * int (x - xc) over the overlap."""
    spec = W._spec(7, 5, (0, 1, 0, 1), 8, 2, np.ones(35), np.zeros(35), q_rects=[(0.13, 0.71, 0.27, 0.93, 2.5)])
    d = Discretisation.from_spec(spec)
    total = np.sum(d.G.reshape(d.nc, 4)[:, 0] * d.cell_int[0])
    assert abs(total - 2.5 * 0.58 * 0.66) < 1e-13
    # x-moment: int_rect x dx dy = 2.5 * 0.66 * (0.71^2 - 0.13^2) / 2 ; recover via basis
    xs_c = (np.arange(d.nc) % d.nx + 0.5) * d.hx
    # eta_1 = sqrt(12/(hx^3 hy)) (x - xc) for the orthonormal basis built from {1, x}
    c1 = d.basis.coef[1, 1]
    mom_x = np.sum(d.G.reshape(d.nc, 4)[:, 1] / c1 + xs_c * d.G.reshape(d.nc, 4)[:, 0] * d.cell_int[0])
    assert abs(mom_x - 2.5 * 0.66 * (0.71 ** 2 - 0.13 ** 2) / 2) < 1e-13


# ---------------------------------------------------------------- DSA (MIP reading)
def test_mip_matrix_spd_and_exact_on_constants_interior():
    """SPD; for per-cell D, the constant function has zero diffusion part in interior rows."""
    d = _small(6, 5)
    A = dsa.mip_matrix(d).toarray()
    assert np.abs(A - A.T).max() < 1e-11 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0
    sig_a = d.sig_t - d.sig_s
    u = d.project_function(lambda x, y: 1.0 + 0 * x)
    Au = A @ u
    for iy in range(1, d.ny - 1):
        for ix in range(1, d.nx - 1):
            c = iy * d.nx + ix
            assert np.abs(Au[4 * c:4 * c + 4] - sig_a[c] * u[4 * c:4 * c + 4]).max() < 1e-11


def test_mip_exact_on_linear_functions_constant_diffusion():
    spec = W._spec(6, 5, (0, 1.2, 0, 1), 8, 2, np.full(30, 2.0), np.full(30, 1.4))
    d = Discretisation.from_spec(spec)
    A = dsa.mip_matrix(d)
    for f in (lambda x, y: 1.0 + 0 * x, lambda x, y: x, lambda x, y: y, lambda x, y: x * y):
        u = d.project_function(f)
        Au = A @ u
        for iy in range(1, d.ny - 1):
            for ix in range(1, d.nx - 1):
                c = iy * d.nx + ix
                assert np.abs(Au[4 * c:4 * c + 4] - 0.6 * u[4 * c:4 * c + 4]).max() < 1e-11


# ---------------------------------------------------------------- low rank (Sec. 3, Alg. 1-2)
def test_mgs2a_orthonormal_hierarchical_and_reconstructs():
    rng = np.random.default_rng(5)
    N = 200
    X = np.zeros((N, 0))
    cols = []
    Rc = []
    for i in range(12):
        v = rng.standard_normal(N) * (10.0 ** (-i % 4))
        if i > 3:
            v = v + X @ rng.standard_normal(X.shape[1]) * 1e3     # nearly dependent snapshots
        x, c, a, failed, _ = lowrank.mgs2a_append(X, v, 1e-10, 4)
        assert not failed
        X_old = X
        X = np.concatenate([X, x[:, None]], axis=1)
        assert np.array_equal(X[:, :-1], X_old)                    # hierarchy X^(k) = [X^(k-1) P]
        cols.append(v)
        Rc.append(np.concatenate([c, [a]]))
    assert np.abs(X.T @ X - np.eye(12)).max() < 1e-13
    R = np.zeros((12, 12))
    for i, c in enumerate(Rc):
        R[:len(c), i] = c
    assert np.abs(X @ R - np.stack(cols, 1)).max() < 1e-9 * np.abs(np.stack(cols, 1)).max()


def test_truncation_tail_rule():
    rng = np.random.default_rng(2)
    s = np.array([10.0, 3.0, 1.0, 1e-6, 1e-9, 1e-12])
    U, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    V, _ = np.linalg.qr(rng.standard_normal((9, 6)))
    C = U @ np.diag(s) @ V.T
    X = np.eye(6)
    for eps, r in ((1e-8, 4), (1e-5, 3), (0.2, 2), (1e-14, 6)):
        Xu, ss, VV = lowrank.truncate(X, C, eps)
        assert len(ss) == r
        assert np.abs(ss - s[:r]).max() < 1e-12


def test_compression_ratio_reproduces_paper_tables():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_compression_ratios.txt"))
            if l.strip() and not l.startswith("#")]
    for name, nx, ny, nt, nz, rank, cr in rows:
        nxd = 4 * int(nx) * int(ny)
        no = int(nt) * int(nz)
        got = 100 * lowrank.compression_ratio(int(rank), nxd, no)
        assert abs(got - float(cr)) < 0.006, name
        assert int(rank) <= no // 2      # rank ceiling from the +-Omega_z twins


def test_lowrank_invariants_and_full_rank_special_case():
    d = _small(5, 4, inflow=(0.2, 0.0, 0.0, 0.3))
    rng = np.random.default_rng(11)
    phi_prev = np.abs(rng.standard_normal(d.ndof))
    trace = []
    out = lowrank.lowrank_si(d, phi_prev, 1, dict(eps_res=1e-13, eps_diff=1e-13, p=1, q=4), trace=trace)
    X = out['X']
    assert np.abs(X.T @ X - np.eye(X.shape[1])).max() < 1e-12
    assert out['rank'] <= d.n_angles // 2
    # when every distinct direction is in the basis, the low-rank SI step is the full-rank one
    assert out['rank'] == d.n_angles // 2
    full = si_dsa.si_step(d, phi_prev)
    assert np.linalg.norm(out['phi'] - full) <= 1e-10 * np.linalg.norm(full)
    # a swept angle's Galerkin solution equals its R column (remark in Sec. 3.2)
    S = d.scattering_source(phi_prev)
    C = out['C']
    for j in np.nonzero(out['swept'])[0][:4]:
        c, _ = lowrank.galerkin_solve(d, X, j, S + d.gbc(j))
        assert np.abs(c - C[:, j]).max() < 1e-9 * max(1, np.abs(c).max())
    # rank grows by at most p per inner iteration (by 0 on a breakdown)
    ranks = [t['rank'] for t in trace]
    assert ranks[0] == 1 and all(0 <= b - a <= 1 for a, b in zip(ranks, ranks[1:]))
    assert out['stats']['mgs_fail'] == 0


def test_lowrank_si_dsa_matches_full_rank_fixed_point():
    d = Discretisation.from_spec(W.random_small(6, 6, n_theta=16, n_omz=2, seed=4))
    phi_c, _ = si_dsa.coupled_direct_solve(d)
    r = lowrank.lowrank_si_dsa(d, dict(eps_si=1e-9, eps_res=1e-10, eps_diff=1e-10, p=1, q=4))
    assert r['converged']
    assert np.linalg.norm(r['phi'] - phi_c) <= 1e-7 * np.linalg.norm(phi_c)


# ---------------------------------------------------------------- adjoint
def test_adjoint_chi_is_transposed_system_solution_and_gradient_matches_fd():
    spec = W.random_small(4, 3, n_theta=8, n_omz=2, seed=9, ratio_range=(0.3, 0.9))
    d = Discretisation.from_spec(spec)
    det = d.rect_functional((0.5, 1.0, 0.4, 1.0))
    phi, _ = si_dsa.coupled_direct_solve(d)
    g = gradients(d, phi, det)
    rng = np.random.default_rng(1)
    h = 1e-6
    for which in ('sig_t', 'sig_s', 'q'):
        v = rng.standard_normal(d.nc)
        vals = []
        for sgn in (+1, -1):
            sp2 = W.random_small(4, 3, n_theta=8, n_omz=2, seed=9, ratio_range=(0.3, 0.9))
            if which == 'sig_t':
                sp2.sig_t = sp2.sig_t + sgn * h * v
            elif which == 'sig_s':
                sp2.sig_s = sp2.sig_s + sgn * h * v
            else:
                sp2.q_cell = sp2.q_cell + sgn * h * v
            d2 = Discretisation.from_spec(sp2)
            vals.append(det @ si_dsa.coupled_direct_solve(d2)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        an = g[which] @ v
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-12), which


def test_gaussian_source_moments_against_closed_forms():
    """Gaussian source exp(-100 (x^2 + y^2)) of Sec. 4.1 on [-1,1]^2: the cell-average moments
    sum to (pi / 100) erf(10)^2, and each cell's x-moment int (x - x_c) q over the cell equals
    the separable closed form [(e^{-100 a^2} - e^{-100 b^2}) / 200 + (0 - x_c) int e] * int_y e
    (the oracle integrates by quadrature; these are the exact integrals)."""
    spec = W.homogeneous_gaussian_e1(1, 1.0, n=7)          # cell edges off the Gaussian's centre
    d = Discretisation.from_spec(spec)
    G = d.G.reshape(d.nc, 4)
    total = np.sum(G[:, 0] * d.cell_int[0])
    assert abs(total - math.pi / 100 * math.erf(10.0) ** 2) < 1e-14
    sq = math.sqrt(math.pi / 100) / 2

    def e_int(a, b):
        return sq * (math.erf(10 * b) - math.erf(10 * a))

    c1 = d.basis.coef[1, 1]                                 # eta_1 = c1 (x - x_c) + ... (orthonormal)
    for iy in range(d.ny):
        for ix in range(d.nx):
            a, b = -1 + ix * d.hx, -1 + (ix + 1) * d.hx
            ya, yb = -1 + iy * d.hy, -1 + (iy + 1) * d.hy
            xc = 0.5 * (a + b)
            ex = (math.exp(-100 * a * a) - math.exp(-100 * b * b)) / 200 - xc * e_int(a, b)
            ref = ex * e_int(ya, yb)
            got = G[iy * d.nx + ix, 1] / c1
            assert abs(got - ref) < 1e-14
            assert abs(G[iy * d.nx + ix, 0] * d.cell_int[0] - e_int(a, b) * e_int(ya, yb)) < 1e-14
