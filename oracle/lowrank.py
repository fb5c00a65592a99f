"""Rank-adaptive low-rank SI and low-rank SI-DSA, Sec. 3.1-3.4, Alg. 1 and Alg. 2.

Oracle (test infrastructure only).  The inner loop of outer iteration n, written in the
order of Sec. 3.1 (steps 1-4) and Sec. 3.3:

  phi_old := phi^{(n-1)};  draw p initial angles at random (Sec. 3.2, "initial sampling")
  for k = 1, 2, ...
    1. sweep the p newly sampled angles (Eq. sampled-sweep)
    2. append each snapshot to X with MGS2-A (Alg. 2), one after the other
    3. draw q unsampled candidate angles at random; Galerkin-solve each
         X^T (D_j + Sigma_t) X c_j = X^T (Sigma_s phi^{(n-1)} + G~_j)   (Eq. galerkin-projection)
       and take the residual r_j = Sigma_s phi^{(n-1)} + G~_j - (D_j + Sigma_t) X c_j
    4. if max_j ||r_j||_2 < eps_res (Eq. residual-chk): Galerkin-solve every angle that has
       no column of R, take the R columns for the appended ones (Sec. 3.2 remark), form
       phi^{(n,k)} = X (C w); stop if ||phi^{(n,k)} - phi_old||_2 <= eps_diff (Eq. phi-diff),
       else phi_old := phi^{(n,k)}
    5. the p candidates with the largest ||r_j||_2 are the next sampled angles
  then the truncated SVD C = U S V^T and X <- X U (Sec. 3.3).

Readings (the paper is silent or ambiguous):
  * the residual uses phi^{(n-1)}, the flux the SI step is solving with (Sec. 3.2 writes phi^{(k)});
  * random draws: each unsampled angle gets a Philox4x32-10 key at (seed, n, k); the q
    (or p, at k = 0) angles with the smallest (key, index) are drawn; if fewer than q
    remain unsampled, all of them are candidates; if none remain, the full check runs
    and the inner loop ends;
  * ties in the residual sort go to the smaller angle index;
  * Alg. 2's orthogonality test is |X(:,1)^T psi_hat| <= eps_MGS as printed (mode 'first');
    mode 'max' tests max_i |X(:,i)^T psi_hat|;  2 mandatory projections + up to m_max = 4
    adaptive ones ("at least 2 and at most 6", Sec. 4);
  * +-Omega_z twins (App. A: the CL rule holds (Ox, Oy, Oz) and (Ox, Oy, -Oz)) have identical
    D_j and g_j^bc in x-y geometry, hence identical psi_j: sweeping angle j samples its twin
    as well (the twin is no longer "unsampled" and reuses j's column of R);
  * breakdown: a snapshot whose orthogonal remainder alpha is <= eps_break * ||psi|| is not
    appended (its angle is marked swept; its C column comes from a Galerkin solve);
  * truncation keeps the smallest r' with sum_{i>r'} s_i / sum_i s_i <= eps_SVD;
  * the outer loop stops on ||phi^{(n,*)} - phi^{(n-1)}||_inf <= eps_SI before the DSA step;
  * basis_update='mgsqr' / 'qr' (Sec. 4.2, Table 2): one projection per snapshot; MGS-QR
    re-orthogonalises the whole basis by a full QR when the test of Alg. 2 fails, QR after
    every inner iteration; the snapshot coefficients R are carried along (stats['full_qr']);
  * sampling='deim' (remark in Sec. 3.2): every inner iteration forms C for all angles and stops
    on the flux change alone; the next p angles are the DEIM points of the p leading right
    singular vectors of C among the unsampled angles (ties to the smaller index);
  * init_angles: a given set of directions replaces the random initial draw of every inner loop
    (Sec. 3.2 leaves the initialisation open to problem-specific strategies; Sec. 3.6 proposes
    initial samples from the previous time step's angular basis in implicit time marching); the
    candidate draws of k >= 1 keep their (seed, n, k) keys.
"""
import numpy as np

from .philox import draw_without_replacement
from .transport import DirectSweeper
from .dsa import MIPSolver


DEFAULTS = dict(eps_si=1e-6, eps_res=1e-7, eps_diff=1e-7, eps_svd=1e-8, eps_mgs=1e-10,
                p=1, q=8, m_max=4, max_outer=100, max_inner=100000, seed=20260101,
                mgs_test='first', eps_break=1e-12, truncate=True, sampling='residual',
                basis_update='mgs2a', init_angles=None)


def full_qr(X, R):
    """Full QR re-orthogonalisation of the basis (the MGS-QR and QR variants of Sec. 4.2):
    X = Q T with diag(T) > 0, X <- Q and the snapshot coefficients R <- T R (the snapshots
    X R are unchanged)."""
    Q, T = np.linalg.qr(X)
    sg = np.where(np.diag(T) < 0, -1.0, 1.0)
    return Q * sg[None, :], (T * sg[:, None]) @ R


def deim_points(V, allowed, p):
    """DEIM index selection (Chaturantabut and Sorensen, 2010) on the columns of V in order,
    restricted to the rows in `allowed`: the first point maximises |V[:, 0]|; point l maximises
    the interpolation residual |V[:, l] - V[:, :l] (V[I, :l]^{-1} V[I, l])| over the allowed rows
    (ties to the smaller row index).  Returns min(p, columns, allowed) points."""
    allowed = np.asarray(sorted(allowed))
    pts = []
    for l in range(min(p, V.shape[1], len(allowed))):
        v = V[:, l]
        if pts:
            c = np.linalg.solve(V[pts, :l], v[pts])
            v = v - V[:, :l] @ c
        a = np.abs(v[allowed])
        pts.append(int(allowed[int(np.argmax(a))]))
    return pts


def mgs2a_append(X, psi, eps_mgs=1e-10, m_max=4, test='first', passes=2):
    """Alg. 2 for one snapshot: returns (new basis vector, c, alpha, failed, n_passes).  `passes`
    mandatory projections (2 in Alg. 2; 1 for the single-MGS variants of Sec. 4.2)."""
    r = X.shape[1]
    ph = np.array(psi, dtype=np.float64)
    c = np.zeros(r)
    mandatory = passes
    passes = 0
    for _ in range(mandatory):
        dc = X.T @ ph
        ph = ph - X @ dc
        c = c + dc
        passes += 1
    alpha = np.linalg.norm(ph)
    if alpha == 0.0:
        return ph, c, 0.0, False, passes
    ph = ph / alpha

    def ortho_err(v):
        if r == 0:
            return 0.0
        if test == 'first':
            return abs(X[:, 0] @ v)
        return np.max(np.abs(X.T @ v))

    for _ in range(m_max):
        if ortho_err(ph) <= eps_mgs:
            break
        ph = alpha * ph
        dc = X.T @ ph
        ph = ph - X @ dc
        c = c + dc
        alpha = np.linalg.norm(ph)
        ph = ph / alpha
        passes += 1
    failed = ortho_err(ph) > eps_mgs
    return ph, c, alpha, failed, passes


def _requalify(X, Rcols):
    """full_qr of the basis with the stored R columns (one per appended angle, shorter ones
    zero-padded) carried along."""
    r = X.shape[1]
    Rm = np.zeros((r, len(Rcols)))
    for i, (_, cv) in enumerate(Rcols):
        Rm[:len(cv), i] = cv
    X, Rm = full_qr(X, Rm)
    return X, [(j, Rm[:, i].copy()) for i, (j, _) in enumerate(Rcols)]


def galerkin_solve(disc, X, j, rhs_j):
    """Eq. (galerkin-projection): c_j = (X^T (D_j+Sigma_t) X)^{-1} X^T rhs_j."""
    LX = disc.L(j) @ X
    A = X.T @ LX
    c = np.linalg.solve(A, X.T @ rhs_j)
    return c, LX


def truncate(X, C, eps_svd):
    """Truncated SVD of C (Sec. 3.3): returns X U, s, V with the tail rule of the header."""
    U, s, Vt = np.linalg.svd(C, full_matrices=False)
    total = s.sum()
    r = len(s)
    if total > 0:
        tail = total - np.cumsum(s)          # tail[i] = sum_{m > i} s_m  (0-based i)
        ok = np.nonzero(tail / total <= eps_svd)[0]
        r = int(ok[0]) + 1 if len(ok) else len(s)
    return X @ U[:, :r], s[:r], Vt[:r].T


def _all_coefficients(disc, X, Rcols, col_of, rhs, M):
    """C of Eq. (lr_for_allangles): the R column of every appended angle (and of its twin), the
    Galerkin solution for every other angle."""
    r = X.shape[1]
    C = np.zeros((r, M))
    rcoef = dict(Rcols)
    for j in range(M):
        if col_of[j] >= 0:
            cv = rcoef[j]
            C[:len(cv), j] = cv
        else:
            C[:, j], _ = galerkin_solve(disc, X, j, rhs(j))
    return C


def twin_map(disc):
    """Index of the ordinate with the same (Omega_x, Omega_y) and opposite Omega_z."""
    tw = np.arange(disc.n_angles)
    for j in range(disc.n_angles):
        m = np.nonzero((np.abs(disc.Ox - disc.Ox[j]) < 1e-14) & (np.abs(disc.Oy - disc.Oy[j]) < 1e-14)
                       & (np.arange(disc.n_angles) != j))[0]
        if len(m):
            tw[j] = m[0]
    return tw


def lowrank_si(disc, phi_prev, n_outer, opts=None, sweeper=None, trace=None, extra=None):
    """One low-rank SI solve (the inner loop of outer iteration n_outer); returns a dict with
    phi (= phi^{(n,*)}), X, C, factors, counters.  `extra` [N_x, N_Omega], when given, is an
    angle-dependent source added to every ordinate's right-hand side (the previous angular flux
    over dt of a backward-Euler step, Sec. 3.7; it must be equal for +-Omega_z twins).  `trace` (a list) receives one record
    per inner iteration: the rank r_k, the candidate set, each candidate's Galerkin
    coefficients c_j and residual vector r_j with its norm, the selection, and whether the
    full check of Sec. 3.3 ran, and the directions swept in that iteration ('sampled')."""
    o = dict(DEFAULTS)
    o.update(opts or {})
    sweeper = sweeper or DirectSweeper(disc)
    M = disc.n_angles
    S = disc.scattering_source(phi_prev)

    def rhs(j):
        b = S + disc.gbc(j)
        return b if extra is None else b + extra[:, j]

    twin = twin_map(disc)
    swept = np.zeros(M, dtype=bool)
    col_of = np.full(M, -1)              # column of R holding the angle's coefficients
    X = np.zeros((disc.ndof, 0))
    Rcols = []                            # list of (angle, coefficient vector)
    phi_old = np.array(phi_prev, dtype=np.float64)
    unsampled = [j for j in range(M)]
    if o['init_angles'] is None:
        new = draw_without_replacement(o['seed'], n_outer, 0, unsampled, o['p'])
    else:
        new = [int(j) for j in o['init_angles']]
        if not new or min(new) < 0 or max(new) >= M:
            raise ValueError("init_angles must be a non-empty list of ordinate indices")
    stats = dict(inner=0, mgs_fail=0, breakdowns=0, full_checks=0, sweeps=0, passes=0)
    phi_k = None
    k = 0
    while True:
        k += 1
        stats['inner'] = k
        sampled = list(new)
        # 1-2: sweep the sampled angles and append them one after the other (Alg. 2)
        for s in new:
            psi = sweeper.sweep(s, S if extra is None else S + extra[:, s])
            stats['sweeps'] += 1
            swept[s] = swept[twin[s]] = True
            if o['basis_update'] == 'mgs2a':
                ph, c, alpha, failed, passes = mgs2a_append(X, psi, o['eps_mgs'], o['m_max'], o['mgs_test'])
            else:
                # MGS-QR and QR (Sec. 4.2, Table 2): a single projection; MGS-QR falls back on a
                # full QR of the basis when the orthogonality test of Alg. 2 fails
                ph, c, alpha, failed, passes = mgs2a_append(X, psi, o['eps_mgs'], 0, o['mgs_test'], passes=1)
            stats['passes'] += passes
            if alpha <= o['eps_break'] * np.linalg.norm(psi):
                stats['breakdowns'] += 1
                continue
            X = np.concatenate([X, ph[:, None]], axis=1)
            col_of[s] = col_of[twin[s]] = X.shape[1] - 1
            Rcols.append((s, np.concatenate([c, [alpha]])))
            if twin[s] != s:
                Rcols.append((twin[s], Rcols[-1][1]))
            if o['basis_update'] == 'mgsqr' and failed:
                X, Rcols = _requalify(X, Rcols)
                stats['full_qr'] = stats.get('full_qr', 0) + 1
            elif o['basis_update'] == 'mgs2a':
                stats['mgs_fail'] += int(failed)
        if o['basis_update'] == 'qr' and X.shape[1] > 0:
            X, Rcols = _requalify(X, Rcols)
            stats['full_qr'] = stats.get('full_qr', 0) + 1
        r = X.shape[1]
        unsampled = [j for j in range(M) if not swept[j]]
        if o['sampling'] == 'deim':
            # DEIM sampling (remark in Sec. 3.2): Galerkin coefficients of every angle (Eq.
            # lr_for_allangles), the flux from them and the stop test on its change, then the SVD
            # C = U S V^T and the DEIM points of the p leading right singular vectors among the
            # unsampled angles (the reading: the residual test needs candidates, which DEIM does not
            # draw, so only the flux-change test of Sec. 3.3 stops the loop)
            C = _all_coefficients(disc, X, Rcols, col_of, rhs, M)
            phi_k = X @ (C @ disc.w)
            dphi = np.linalg.norm(phi_k - phi_old)
            stats['full_checks'] += 1
            rec = dict(k=k, rank=r, phi_diff=dphi, full_check=True, sampled=sampled)
            stop = dphi <= o['eps_diff'] or not unsampled
            if not stop:
                phi_old = phi_k
                _, sv, Vt = np.linalg.svd(C, full_matrices=False)
                rec['selected'] = deim_points(Vt.T, unsampled, o['p'])
                rec['singular_values'] = sv
            if trace is not None:
                trace.append(rec)
            if stop or k >= o['max_inner']:
                break
            new = rec['selected']
            continue
        # 3: random candidates and their Galerkin residuals
        cand = draw_without_replacement(o['seed'], n_outer, k, unsampled, o['q'])
        norms, resid, coef = [], [], []
        for j in cand:
            c, LX = galerkin_solve(disc, X, j, rhs(j))
            rj = rhs(j) - LX @ c
            norms.append(np.linalg.norm(rj))
            resid.append(rj)
            coef.append(c)
        norms = np.array(norms)
        order = sorted(range(len(cand)), key=lambda i: (-norms[i], cand[i]))
        selected = [cand[i] for i in order[:o['p']]]
        rec = dict(k=k, rank=r, candidates=list(cand), norms=norms.copy(), selected=selected,
                   residuals=resid, coefficients=coef, full_check=False, sampled=sampled)
        # 4: stopping test (Sec. 3.3)
        stop = False
        if len(cand) == 0 or norms.max() < o['eps_res']:
            stats['full_checks'] += 1
            rec['full_check'] = True
            C = _all_coefficients(disc, X, Rcols, col_of, rhs, M)
            phi_k = X @ (C @ disc.w)
            dphi = np.linalg.norm(phi_k - phi_old)
            rec['phi_diff'] = dphi
            if dphi <= o['eps_diff'] or len(cand) == 0:
                stop = True
            else:
                phi_old = phi_k
        if trace is not None:
            trace.append(rec)
        if stop or k >= o['max_inner']:
            break
        new = selected
    out = dict(phi=phi_k, X=X, C=C, rank=X.shape[1], stats=stats, swept=swept)
    if o['truncate']:
        Xu, s, V = truncate(X, C, o['eps_svd'])
        out.update(U_X=Xu, S=s, V=V, rank_trunc=len(s))
    return out


def lowrank_si_dsa(disc, opts=None, phi0=None, sweeper=None, mip=None, trace=None, extra=None):
    """Alg. 1: low-rank SI followed by the DSA correction until the outer stop test holds
    (`extra`: see lowrank_si)."""
    o = dict(DEFAULTS)
    o.update(opts or {})
    sweeper = sweeper or DirectSweeper(disc)
    mip = mip or MIPSolver(disc)
    phi = np.zeros(disc.ndof) if phi0 is None else np.array(phi0, dtype=np.float64)
    diffs, ranks, inner = [], [], []
    last = None
    converged = False
    n = 0
    for n in range(1, o['max_outer'] + 1):
        t = [] if trace is not None else None
        last = lowrank_si(disc, phi, n, o, sweeper, t, extra)
        if trace is not None:
            trace.append(t)
        phi_star = last['phi']
        diffs.append(np.max(np.abs(phi_star - phi)))
        ranks.append(last['rank'])
        inner.append(last['stats']['inner'])
        if diffs[-1] <= o['eps_si']:
            phi = phi_star
            converged = True
            break
        phi = phi_star + mip.correction(phi_star, phi)
    return dict(phi=phi, iters=n, diffs=diffs, ranks=ranks, inner=inner, last=last,
                converged=converged)


def compression_ratio(rank, n_x, n_omega):
    """DOFs of X, V and the diagonal S over those of the full Psi (Sec. 4 metrics)."""
    return rank * (n_x + n_omega + 1) / (n_x * n_omega)
