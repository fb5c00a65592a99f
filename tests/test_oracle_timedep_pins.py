"""Pins of the oracle's backward-Euler step (Sec. 3.7) against values fixed by mathematics:
closed forms of the homogeneous medium, the steady limit, particle balance over a step, and
the equivalence of the mass-matrix modification with a shifted sigma_t.  CPU only."""
import math

import numpy as np

import workloads as W
from oracle import si_dsa, timedep
from oracle.dg import Discretisation


def _const(d, c):
    """The coefficient vector of the constant c on every cell (orthonormal basis)."""
    v = np.zeros(d.ndof)
    v[0::4] = c * math.sqrt(d.hx * d.hy)
    return v


def test_step_operator_is_the_total_cross_section_shifted_by_one_over_dt():
    """The mass matrix of the orthonormal basis is the identity, so D_j + Sigma_t + M/dt is the
    operator of sigma_t + 1/dt in every cell."""
    spec = W.random_small(5, 4, n_theta=8, n_omz=2, seed=3)
    d = Discretisation.from_spec(spec)
    dt = 0.37
    ds = Discretisation.from_spec(spec, sig_t=spec.sig_t + 1.0 / dt)
    assert abs(timedep.global_mass(d) - np.eye(d.ndof)).max() < 1e-14
    for j in (0, 5, 11):
        diff = timedep.step_operator(d, j, dt) - ds.L(j)
        assert abs(diff).max() < 1e-13


def test_homogeneous_medium_steps_follow_the_closed_form():
    """Constant medium, constant isotropic psi^0 = c0 and inflow equal to the exact next value:
    every step keeps psi constant, c_{n+1} = (c_n / dt + q) / (1 / dt + sigma_a) (the backward
    Euler step of the infinite-medium balance), for the coupled solve and the SI-DSA."""
    sig_t, sig_s, q, dt, c0 = 2.0, 1.5, 1.0, 0.3, 0.2
    c = c0
    for step in range(2):
        c_next = (c / dt + q) / (1.0 / dt + (sig_t - sig_s))
        spec = W.infinite_medium(5, 4, sig_t, sig_s, q, n_theta=8, n_omz=2, box=(0.0, 1.3, -0.2, 0.7))
        spec.inflow = (c_next,) * 4
        d = Discretisation.from_spec(spec)
        psi0 = np.tile(_const(d, c)[:, None], (1, d.n_angles))
        phi, psi = timedep.be_coupled_solve(d, psi0, dt)
        exact = _const(d, c_next)
        assert np.abs(phi - exact).max() < 1e-12
        assert np.abs(psi - exact[:, None]).max() < 1e-12
        r = timedep.be_si_dsa(spec, psi0, dt, eps_si=1e-14, max_iter=300)
        assert r['converged'] and np.abs(r['phi'] - exact).max() < 1e-12
        c = c_next
    # the marching keeps approaching the steady value q / sigma_a
    assert c0 < c < q / (sig_t - sig_s)


def test_angle_dependent_initial_flux_in_the_deep_interior():
    """Spatially constant but angle-dependent psi^0_j: away from the boundary (inflow effects
    decay like exp(-(sigma_t + 1/dt) distance), here below 1e-30) each ordinate follows its own
    closed form  phi^1 = (q + phi^0/dt)/(1/dt + sigma_a),
    psi^1_j = (sigma_s phi^1 + q + psi^0_j/dt)/(1/dt + sigma_t)  -- which fails if an ordinate
    receives another ordinate's source."""
    sig_t, sig_s, q, dt = 1.0, 0.6, 0.5, 0.004
    n = 24
    spec = W._spec(n, n, (0, 1, 0, 1), 8, 2, np.full(n * n, sig_t), np.full(n * n, sig_s),
                   q_cell=np.full(n * n, q))
    d = Discretisation.from_spec(spec)
    f = 1.0 + 0.5 * d.Ox + 0.25 * d.Oy ** 2 + 0.1 * d.Oz
    psi0 = np.outer(_const(d, 1.0), f)
    phi0 = float(f @ d.w)
    phi1 = (q + phi0 / dt) / (1.0 / dt + sig_t - sig_s)
    psi1 = (sig_s * phi1 + q + f / dt) / (1.0 / dt + sig_t)
    _, psi = timedep.be_coupled_solve(d, psi0, dt)
    unit = math.sqrt(d.hx * d.hy)
    for iy in range(8, 16):
        for ix in range(8, 16):
            c = iy * n + ix
            # rounding of the coupled LU (entries ~ 1/dt = 250) leaves a few 1e-10; a source
            # taken from another ordinate would be off by ~0.1
            assert np.abs(psi[4 * c, :] / unit - psi1).max() < 1e-8 * psi1.max()
            assert np.abs(psi[4 * c + 1:4 * c + 4, :]).max() < 1e-8 * psi1.max()


def test_large_dt_reduces_to_the_steady_solution():
    spec = W.random_small(6, 5, n_theta=8, n_omz=2, seed=4, inflow=(0.3, 0.0, 0.2, 0.1))
    d = Discretisation.from_spec(spec)
    rng = np.random.default_rng(5)
    psi0 = rng.standard_normal((d.ndof, d.n_angles))
    phi_s, psi_s = si_dsa.coupled_direct_solve(d)
    phi, psi = timedep.be_coupled_solve(d, psi0, 1e14)
    assert np.linalg.norm(phi - phi_s) <= 1e-9 * np.linalg.norm(phi_s)
    assert np.linalg.norm(psi - psi_s) <= 1e-9 * np.linalg.norm(psi_s)


def test_particle_balance_over_a_step():
    """Over one step: (total particles at n+1 - at n)/dt + leakage + absorption = source + inflow
    (test function eta = 1, summed over ordinates)."""
    spec = W.random_small(6, 5, n_theta=8, n_omz=2, seed=6, inflow=(0.5, 0.0, 1.0, 0.25))
    d = Discretisation.from_spec(spec)
    rng = np.random.default_rng(7)
    psi0 = np.abs(rng.standard_normal((d.ndof, d.n_angles)))
    dt = 0.05
    phi, psi = timedep.be_coupled_solve(d, psi0, dt)
    b = d.basis
    ys, wy = b.vface_quad()
    xs, wx = b.hface_quad()
    vR, _, _ = b.eval(np.full_like(ys, d.hx / 2), ys)
    vL, _, _ = b.eval(np.full_like(ys, -d.hx / 2), ys)
    vT, _, _ = b.eval(xs, np.full_like(xs, d.hy / 2))
    vB, _, _ = b.eval(xs, np.full_like(xs, -d.hy / 2))
    gL, gR, gB, gT = d.inflow
    leak = inflow = 0.0
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
    total = lambda ph: np.sum(ph.reshape(d.nc, 4) @ d.cell_int)
    absorption = np.sum((d.sig_t - d.sig_s) * (phi.reshape(d.nc, 4) @ d.cell_int))
    source = np.sum(d.G.reshape(d.nc, 4)[:, 0] * d.cell_int[0])
    change = (total(phi) - total(psi0 @ d.w)) / dt
    assert abs(change + leak + absorption - source - inflow) < 1e-11 * (abs(change) + source + inflow)


def test_step_si_dsa_reaches_the_coupled_solution():
    spec = W.random_small(6, 5, n_theta=8, n_omz=2, seed=8, ratio_range=(0.8, 0.99))
    d = Discretisation.from_spec(spec)
    rng = np.random.default_rng(9)
    psi0 = np.abs(rng.standard_normal((d.ndof, d.n_angles)))
    phi_c, psi_c = timedep.be_coupled_solve(d, psi0, 0.5)
    r = timedep.be_si_dsa(spec, psi0, 0.5, eps_si=1e-13, max_iter=500)
    r0 = timedep.be_si_dsa(spec, psi0, 0.5, eps_si=1e-13, max_iter=2000, use_dsa=False)
    assert r['converged'] and r0['converged']
    assert np.linalg.norm(r['phi'] - phi_c) <= 1e-10 * np.linalg.norm(phi_c)
    assert np.linalg.norm(r['psi'] - psi_c) <= 1e-10 * np.linalg.norm(psi_c)
    assert np.linalg.norm(r0['phi'] - phi_c) <= 1e-10 * np.linalg.norm(phi_c)
    assert r['iters'] < r0['iters']


def _twin_symmetric(d, psi):
    """psi with each +-Omega_z twin pair set to the pair's mean (low-rank steps need it)."""
    from oracle.lowrank import twin_map
    tw = twin_map(d)
    return 0.5 * (psi + psi[:, tw])


def test_lowrank_step_homogeneous_closed_form_at_rank_one():
    """The low-rank step of the homogeneous problem (constant psi^0 = c0, inflow at the exact
    next value) returns the constant c1 = (c0/dt + q)/(1/dt + sigma_a), from a rank-1 basis in
    its last outer iteration."""
    sig_t, sig_s, q, dt, c0 = 2.0, 1.5, 1.0, 0.3, 0.2
    c1 = (c0 / dt + q) / (1.0 / dt + (sig_t - sig_s))
    spec = W.infinite_medium(5, 4, sig_t, sig_s, q, n_theta=8, n_omz=2, box=(0.0, 1.3, -0.2, 0.7))
    spec.inflow = (c1,) * 4
    d = Discretisation.from_spec(spec)
    psi0 = np.tile(_const(d, c0)[:, None], (1, d.n_angles))
    # the exact solution's residuals are rounding (~1e-14): any tolerance above that stops at rank 1
    r = timedep.be_lowrank(spec, psi0, dt, dict(eps_si=1e-12, eps_res=1e-10, eps_diff=1e-10, p=1, q=4, seed=3))
    exact = _const(d, c1)
    # early outer iterations (phi^(0) = 0) are not constant; once phi has converged each SI step's
    # solution is the constant, found with one sampled ordinate
    assert r['converged'] and r['ranks'][-1] == 1
    assert np.abs(r['phi'] - exact).max() < 1e-12
    assert np.abs(r['psi'] - exact[:, None]).max() < 1e-12


def test_lowrank_step_reaches_the_coupled_solution_of_the_step():
    """At tight tolerances the low-rank step's fixed point is the step's coupled solution."""
    spec = W.random_small(6, 5, n_theta=8, n_omz=2, seed=10, inflow=(0.2, 0.1, 0.0, 0.3))
    d = Discretisation.from_spec(spec)
    rng = np.random.default_rng(11)
    psi0 = _twin_symmetric(d, np.abs(rng.standard_normal((d.ndof, d.n_angles))))
    dt = 0.4
    phi_c, psi_c = timedep.be_coupled_solve(d, psi0, dt)
    r = timedep.be_lowrank(spec, psi0, dt, dict(eps_si=1e-12, eps_res=1e-12, eps_diff=1e-12, p=2, q=6, seed=4))
    assert r['converged']
    assert np.linalg.norm(r['phi'] - phi_c) <= 1e-9 * np.linalg.norm(phi_c)
    assert np.linalg.norm(r['psi'] - psi_c) <= 1e-8 * np.linalg.norm(psi_c)


# Warm-started sampling of the low-rank steps (the combination Sec. 3.6 proposes for implicit
# time marching: initial samples from the previous step's angular basis by DEIM).

def test_initial_angles_equal_to_the_random_draw_reproduce_the_cold_start():
    """init_angles only replaces the initial draw: given the very angles the (seed, n, 0) draw
    picks, the inner loop is the cold one, bit for bit."""
    from oracle import lowrank
    from oracle.philox import draw_without_replacement
    spec = W.random_small(5, 4, n_theta=8, n_omz=2, seed=12, inflow=(0.2, 0.0, 0.1, 0.3))
    d = Discretisation.from_spec(spec)
    phi_prev = np.random.default_rng(13).standard_normal(d.ndof)
    opts = dict(eps_res=1e-9, eps_diff=1e-9, p=2, q=5, seed=7)
    cold = lowrank.lowrank_si(d, phi_prev, 3, opts)
    init = draw_without_replacement(7, 3, 0, list(range(d.n_angles)), 2)
    t = []
    warm = lowrank.lowrank_si(d, phi_prev, 3, dict(opts, init_angles=init), trace=t)
    assert t[0]['sampled'] == list(init)
    assert np.array_equal(cold['phi'], warm['phi']) and np.array_equal(cold['X'], warm['X'])
    assert cold['stats'] == warm['stats']


def _diffusive_spec(n=6):
    """Homogeneous, scattering-dominated medium (sigma_t = 10, c = 0.99) with a centred source and
    vacuum boundaries: an angular flux of low numerical rank."""
    return W._spec(n, n, (0, 1, 0, 1), 16, 4, np.full(n * n, 10.0), np.full(n * n, 9.9),
                   q_rects=[(0.3, 0.7, 0.3, 0.7, 1.0)])


def test_warm_started_step_starts_every_inner_loop_from_the_deim_points_of_the_previous_basis():
    from oracle.lowrank import twin_map
    spec = _diffusive_spec()
    d = Discretisation.from_spec(spec)
    opts = dict(eps_si=1e-6, eps_res=3e-4, eps_diff=3e-4, eps_svd=1e-4, p=1, q=4, seed=11)
    first = timedep.be_lowrank(spec, np.zeros((d.ndof, d.n_angles)), 1.0, opts)
    V = first['V']
    assert V.shape[0] == d.n_angles                      # right singular vectors: one row per ordinate
    tr = []
    second = timedep.be_lowrank(spec, first['psi'], 1.0, opts, trace=tr, warm_V=V)
    init = second['init_angles']
    twin = twin_map(d)
    # the defining properties of a DEIM set of V: r' distinct directions, one per twin pair at most,
    # and V restricted to them nonsingular (the interpolation is well posed)
    assert len(init) == V.shape[1] < d.n_angles // 2
    assert len(set(init)) == len(init) and not any(twin[j] in init and twin[j] != j for j in init)
    assert np.linalg.matrix_rank(V[init, :]) == V.shape[1]
    assert init == timedep.warm_start_angles(d, V)
    for outer in tr:                                     # every inner loop of the step
        assert outer[0]['sampled'] == init
    # the greedy loop goes on from the warm set where the residuals ask for it
    assert max(second['inner']) > 1 and second['converged']


def test_warm_started_step_reaches_the_coupled_solution_of_the_step():
    spec = W.random_small(6, 5, n_theta=8, n_omz=2, seed=10, inflow=(0.2, 0.1, 0.0, 0.3))
    d = Discretisation.from_spec(spec)
    rng = np.random.default_rng(11)
    psi0 = _twin_symmetric(d, np.abs(rng.standard_normal((d.ndof, d.n_angles))))
    dt = 0.4
    tight = dict(eps_si=1e-12, eps_res=1e-12, eps_diff=1e-12, p=2, q=6, seed=4)
    prev = timedep.be_lowrank(spec, psi0, dt, dict(tight, eps_si=1e-6, eps_res=1e-6, eps_diff=1e-6))
    phi_c, psi_c = timedep.be_coupled_solve(d, prev['psi'], dt)
    r = timedep.be_lowrank(spec, prev['psi'], dt, tight, warm_V=prev['V'])
    assert r['converged'] and r['init_angles'] is not None
    assert np.linalg.norm(r['phi'] - phi_c) <= 1e-9 * np.linalg.norm(phi_c)
    assert np.linalg.norm(r['psi'] - psi_c) <= 1e-8 * np.linalg.norm(psi_c)


def test_warm_started_homogeneous_step_keeps_the_closed_form_at_rank_one():
    sig_t, sig_s, q, dt, c0 = 2.0, 1.5, 1.0, 0.3, 0.2
    c1 = (c0 / dt + q) / (1.0 / dt + (sig_t - sig_s))
    c2 = (c1 / dt + q) / (1.0 / dt + (sig_t - sig_s))
    spec = W.infinite_medium(5, 4, sig_t, sig_s, q, n_theta=8, n_omz=2, box=(0.0, 1.3, -0.2, 0.7))
    d = Discretisation.from_spec(spec)
    opts = dict(eps_si=1e-12, eps_res=1e-10, eps_diff=1e-10, p=1, q=4, seed=3)
    spec.inflow = (c1,) * 4
    r1 = timedep.be_lowrank(spec, np.tile(_const(d, c0)[:, None], (1, d.n_angles)), dt, opts)
    assert r1['V'].shape[1] == 1
    spec.inflow = (c2,) * 4
    r2 = timedep.be_lowrank(spec, r1['psi'], dt, opts, warm_V=r1['V'])
    assert len(r2['init_angles']) == 1 and r2['converged']
    assert np.abs(r2['phi'] - _const(d, c2)).max() < 1e-12
    assert np.abs(r2['psi'] - _const(d, c2)[:, None]).max() < 1e-12


def test_warm_start_cuts_the_inner_iterations_of_a_march_at_equal_error():
    """Two steps of the diffusive problem: the second step's inner loops start from the first
    step's basis and need far fewer iterations, and both marches stay as close to the coupled
    march as their tolerances allow."""
    spec = _diffusive_spec()
    d = Discretisation.from_spec(spec)
    psi0 = np.zeros((d.ndof, d.n_angles))
    opts = dict(eps_si=1e-6, eps_res=3e-4, eps_diff=3e-4, eps_svd=1e-4, p=1, q=4, seed=11)
    cold = timedep.be_march_lowrank(spec, psi0, 1.0, 2, opts, warm=False)
    warm = timedep.be_march_lowrank(spec, psi0, 1.0, 2, opts, warm=True)
    ref = timedep.be_march(spec, psi0, 1.0, 2)
    assert warm[0]['init_angles'] is None and warm[1]['init_angles'] is not None
    assert np.array_equal(cold[0]['phi'], warm[0]['phi'])
    assert sum(warm[1]['inner']) * 4 < sum(cold[1]['inner'])
    for i in range(2):
        for r in (cold[i], warm[i]):
            assert r['converged']
            assert np.linalg.norm(r['phi'] - ref[i][0]) <= 1e-4 * np.linalg.norm(ref[i][0])
