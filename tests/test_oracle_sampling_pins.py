"""Pins of the oracle's residual-based greedy sampling (Sec. 3.2) and inner stopping test
(Sec. 3.3) against what the mathematics and the paper's statement fix, independently of the
oracle's own sort and stop code.  CPU only.

  * Galerkin orthogonality: the candidate residual r_j = S + g_j - (D_j + Sigma_t) X c_j of
    the Galerkin coefficients c_j (Eq. galerkin-projection) satisfies X^T r_j = 0.
  * In-span candidates: where every ordinate's exact angular flux lies in span(X) (the infinite
    medium, whose exact S_N-DG solution is the same constant for every ordinate), every
    candidate residual vanishes, and the inner loop ends after its first full check.
  * Residual = operator image of the Galerkin error: r_j = (D_j + Sigma_t)(psi_j - X c_j), with
    psi_j the direct solve of the ordinate's own system.
  * Selection: the p selected candidates carry the p LARGEST residual norms (the descending
    sort of Sec. 3.2; ties to the smaller angle index).
  * Stop test: the full check runs exactly in the inner iterations whose largest candidate
    residual norm is below eps_res (Eq. residual-chk); the loop stops at the first full check
    whose scalar-flux change is within eps_diff (Eq. phi-diff).
"""
import math

import numpy as np

import workloads as W
from oracle import lowrank
from oracle.dg import Discretisation
from oracle.transport import DirectSweeper


def _diffusive():
    """Homogeneous, optically thick, nearly pure scatterer (8 x 8 cells, CL(16,4)): the candidate
    residuals decay gradually, so the trace holds full checks that do and do not stop, and
    inner iterations whose smallest residual is below eps_res while the largest is not."""
    n = 8
    spec = W._spec(n, n, (0, 1, 0, 1), 16, 4, np.full(n * n, 50.0), np.full(n * n, 49.9), q_cell=np.ones(n * n))
    return Discretisation.from_spec(spec)


OPTS = dict(eps_res=1e-3, eps_diff=1e-3, p=2, q=6, seed=5)


def _run(d, phi_prev, opts):
    trace = []
    out = lowrank.lowrank_si(d, phi_prev, 1, opts, trace=trace)
    return out, trace


def test_candidate_residuals_are_galerkin_orthogonal_to_the_basis():
    d = _diffusive()
    out, trace = _run(d, np.zeros(d.ndof), OPTS)
    S = d.scattering_source(np.zeros(d.ndof))
    n_checked = 0
    for rec in trace:
        X = out['X'][:, :rec['rank']]                 # hierarchical basis: the first r_k columns
        for j, rj, nrm in zip(rec['candidates'], rec['residuals'], rec['norms']):
            rhs = S + d.gbc(j)
            assert np.abs(X.T @ rj).max() <= 1e-12 * np.linalg.norm(rhs)
            assert abs(np.linalg.norm(rj) - nrm) <= 1e-14 * max(nrm, 1.0)
            n_checked += 1
    assert n_checked >= 30


def test_candidate_residual_is_the_operator_image_of_the_galerkin_error():
    """r_j = L_j (psi_j - X c_j) with psi_j = L_j^{-1}(S + g_j) from a direct solve: the residual
    measures the candidate's Galerkin error (a residual formed from the right-hand side alone,
    or without the Galerkin term, fails this)."""
    d = _diffusive()
    out, trace = _run(d, np.zeros(d.ndof), OPTS)
    S = d.scattering_source(np.zeros(d.ndof))
    sw = DirectSweeper(d)
    for rec in trace[:4]:
        X = out['X'][:, :rec['rank']]
        for j, rj, cj in zip(rec['candidates'], rec['residuals'], rec['coefficients']):
            psi = sw.sweep(j, S)
            err_img = d.L(j) @ (psi - X @ cj)
            assert np.abs(err_img - rj).max() <= 1e-10 * max(1.0, np.abs(rj).max())
            assert np.linalg.norm(psi - X @ cj) > 0.0 and np.linalg.norm(rj) > 0.0


def test_candidates_whose_flux_is_in_the_span_have_zero_residual():
    """Infinite medium at its exact fixed point: psi_j = q / sigma_a for every ordinate, so one
    sampled ordinate spans every candidate's flux.  All residuals vanish to round-off (while
    the right-hand sides do not), the first inner iteration runs the full check and stops, and
    the flux is the exact constant."""
    spec = W.infinite_medium(5, 4, 2.0, 1.5, 1.0, n_theta=8, n_omz=2)
    d = Discretisation.from_spec(spec)
    exact = np.zeros(d.ndof)
    exact[0::4] = (1.0 / 0.5) * math.sqrt(d.hx * d.hy)
    S = d.scattering_source(exact)
    out, trace = _run(d, exact, dict(eps_res=1e-9, eps_diff=1e-9, p=1, q=4, seed=3))
    assert len(trace) == 1 and trace[0]['rank'] == 1 and trace[0]['full_check']
    for j, rj in zip(trace[0]['candidates'], trace[0]['residuals']):
        assert np.linalg.norm(S + d.gbc(j)) > 1.0
        assert np.linalg.norm(rj) < 1e-12
    assert np.abs(out['phi'] - exact).max() < 1e-12


def test_selected_candidates_carry_the_largest_residual_norms():
    d = _diffusive()
    _, trace = _run(d, np.zeros(d.ndof), OPTS)
    p = OPTS['p']
    n_strict = 0
    for rec in trace:
        norms = np.asarray(rec['norms'])
        cand = list(rec['candidates'])
        if not cand:
            continue
        sel = rec['selected']
        assert len(sel) == min(p, len(cand)) and len(set(sel)) == len(sel) and set(sel) <= set(cand)
        sel_norms = sorted((norms[cand.index(j)] for j in sel), reverse=True)
        rest = [norms[i] for i, j in enumerate(cand) if j not in sel]
        if rest:
            assert min(sel_norms) >= max(rest)
            n_strict += int(min(sel_norms) > max(rest) * (1 + 1e-12))
        # ties to the smaller angle index: the k-th selected has the k-th largest (norm, -index)
        order = sorted(range(len(cand)), key=lambda i: (-norms[i], cand[i]))
        assert sel == [cand[i] for i in order[:len(sel)]]
    assert n_strict >= 5


def test_full_check_runs_exactly_when_the_largest_residual_is_below_eps_res():
    d = _diffusive()
    out, trace = _run(d, np.zeros(d.ndof), OPTS)
    eps_res, eps_diff = OPTS['eps_res'], OPTS['eps_diff']
    mixed = 0
    for rec in trace:
        norms = np.asarray(rec['norms'])
        below = len(norms) == 0 or norms.max() < eps_res
        assert rec['full_check'] == below
        mixed += int(len(norms) > 0 and norms.min() < eps_res <= norms.max())
    # the case holds inner iterations that a smallest-residual test would have stopped on
    assert mixed >= 1
    checks = [rec for rec in trace if rec['full_check']]
    assert len(checks) >= 2
    # every full check but the last saw a flux change above eps_diff; the last one stopped
    assert all(rec['phi_diff'] > eps_diff for rec in checks[:-1])
    assert checks[-1]['phi_diff'] <= eps_diff and trace[-1] is checks[-1]
    assert out['stats']['full_checks'] == len(checks)



def test_fully_greedy_sampling_takes_every_unsampled_angle_as_a_candidate():
    """The fully greedy variant (remark in Sec. 3.2): with q at least the number of angles, the
    first candidate set is every angle but the p initial ones and their +-Omega_z twins (App. A:
    (Ox, Oy, Oz) and (Ox, Oy, -Oz)), each later set is the previous one less the angles selected
    from it and their twins, and the p selected carry the largest residuals of the set."""
    d = _diffusive()
    _, trace = _run(d, np.zeros(d.ndof), dict(OPTS, q=10_000))
    M, p = d.n_angles, OPTS['p']

    def twin(j):
        m = [i for i in range(M) if i != j and abs(d.Ox[i] - d.Ox[j]) < 1e-14 and abs(d.Oy[i] - d.Oy[j]) < 1e-14]
        assert len(m) == 1 and abs(d.Oz[m[0]] + d.Oz[j]) < 1e-14
        return m[0]

    cand = set(trace[0]['candidates'])
    assert len(cand) == M - 2 * p                     # the initial p and their twins are sampled
    for a, b in zip(trace, trace[1:]):
        norms = np.asarray(a['norms'])
        top = sorted(zip(-norms, a['candidates']))[:p]
        assert a['selected'] == [j for _, j in top]
        cand -= set(a['selected']) | {twin(j) for j in a['selected']}
        assert set(b['candidates']) == cand
    # the full check then runs only once the largest residual over every unsampled angle is small
    assert trace[-1]['full_check'] and (len(trace[-1]['norms']) == 0 or max(trace[-1]['norms']) < OPTS['eps_res'])


def test_deim_points_definition_cases():
    """DEIM (Chaturantabut and Sorensen): on columns that are unit vectors e_{i_l} (plus a smaller
    tail) the points are the i_l in order; the points do not change when columns are scaled or
    flipped in sign; and they come from the allowed rows only."""
    rng = np.random.default_rng(3)
    n, idx = 40, [7, 31, 2, 18]
    V = 1e-3 * rng.standard_normal((n, 4))
    for l, i in enumerate(idx):
        V[i, l] += 1.0
    assert lowrank.deim_points(V, range(n), 4) == idx
    Q, _ = np.linalg.qr(rng.standard_normal((n, 5)))
    base = lowrank.deim_points(Q, range(n), 5)
    assert lowrank.deim_points(Q * np.array([3.0, -0.5, 7.0, -2.0, 1e-3]), range(n), 5) == base
    allowed = [i for i in range(n) if i % 3]
    pts = lowrank.deim_points(Q, allowed, 5)
    assert len(set(pts)) == 5 and set(pts) <= set(allowed)
    # the interpolation at the chosen points is exact on the columns used
    P = np.array(pts)
    assert abs(np.linalg.det(Q[P][:, :5])) > 1e-6


def test_deim_sampling_reaches_the_coupled_fixed_point():
    """DEIM sampling inside the low-rank SI-DSA (Alg. 1): the converged flux is the S_N-DG fixed
    point (the direct solve of the coupled system)."""
    from oracle import si_dsa
    d = Discretisation.from_spec(W.random_small(6, 6, n_theta=16, n_omz=2, seed=4))
    phi_c, _ = si_dsa.coupled_direct_solve(d)
    r = lowrank.lowrank_si_dsa(d, dict(eps_si=1e-9, eps_res=1e-10, eps_diff=1e-10, p=2, q=4, sampling='deim'))
    assert r['converged']
    assert np.linalg.norm(r['phi'] - phi_c) <= 1e-7 * np.linalg.norm(phi_c)


def test_full_qr_keeps_the_snapshots_and_orthonormalises():
    """full_qr (Sec. 4.2's MGS-QR / QR variants): X R is unchanged, the new basis is orthonormal
    and the triangular factor has a positive diagonal (Q unique)."""
    rng = np.random.default_rng(8)
    X, _ = np.linalg.qr(rng.standard_normal((60, 7)))
    X = X + 1e-6 * rng.standard_normal(X.shape)          # lost orthogonality
    R = np.triu(rng.standard_normal((7, 9)))
    Q, R2 = lowrank.full_qr(X, R)
    assert np.abs(Q.T @ Q - np.eye(7)).max() < 1e-14
    assert np.abs(Q @ R2 - X @ R).max() < 1e-13 * np.abs(X @ R).max()
    _, T = np.linalg.qr(X)
    assert np.all(np.abs(np.diag(np.linalg.lstsq(Q, X, rcond=None)[0])) > 0)
    assert np.allclose(np.abs(np.diag(np.linalg.lstsq(Q, X, rcond=None)[0])), np.abs(np.diag(T)))


def test_basis_update_variants_give_the_same_step():
    """MGS2-A, MGS-QR and QR build bases of the same span from the same snapshots (Sec. 4.2:
    equal ranks and fluxes up to rounding); QR re-orthogonalises after every inner iteration and
    MGS2-A never.  One angle a step: with p > 1 a +-Omega_z twin pair can be sampled together, and
    after a single projection the second twin's rounding remainder may pass the breakdown test as
    a noise column (the variants' own weakness, not a difference of the spans)."""
    d = _diffusive()
    outs = {bu: _run(d, np.zeros(d.ndof), dict(OPTS, p=1, eps_res=1e-6, eps_diff=1e-6, mgs_test='max',
                                                basis_update=bu))
            for bu in ('mgs2a', 'mgsqr', 'qr')}
    ref = outs['mgs2a'][0]
    for bu, (out, trace) in outs.items():
        assert out['rank'] == ref['rank'] and out['stats']['inner'] == ref['stats']['inner']
        assert np.linalg.norm(out['phi'] - ref['phi']) <= 1e-10 * np.linalg.norm(ref['phi'])
        X = out['X']
        # orthogonality within the test's threshold eps_MGS = 1e-10 (the all-column test of Alg. 2)
        assert np.abs(X.T @ X - np.eye(X.shape[1])).max() < 1e-10
    assert outs['qr'][0]['stats']['full_qr'] == outs['qr'][0]['stats']['inner']
    assert outs['mgs2a'][0]['stats'].get('full_qr', 0) == 0
