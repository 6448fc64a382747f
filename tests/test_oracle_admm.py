"""Pins of the oracle's row reduction, y-solve, Algorithm 1 and certificate — CPU only.

The whole-solve pins compare the relaxation optimum p*_kappa with a brute-force
search of the nonconvex problem (Theorem 1: p*_kappa <= p*, with equality when
every moment matrix has rank one) on horizons 2 and 3.
"""
import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

import workloads as wl
from oracle import certify as CE
from oracle import relax as R
from oracle import sgs_admm as O

from test_oracle_relax import _pend_rollout, _toy_rollout


def test_reduction_rank_and_spd():
    for p in (wl.toy_problem(N=3), wl.pendulum_problem(N=3, theta0=0.1)):
        sdp = R.relax(p)
        keep, _ = O.reduce_rows(sdp)
        Ad = sdp.A.toarray()
        rank = np.linalg.matrix_rank(Ad, tol=1e-9 * np.linalg.norm(Ad, 2))
        assert keep.sum() == rank
        Ak = Ad[keep]
        assert np.min(np.linalg.eigvalsh(Ak @ Ak.T)) > 1e-10
        # every dropped row lies in the span of the kept rows
        drop = Ad[~keep]
        if len(drop):
            coef = np.linalg.lstsq(Ak.T, drop.T, rcond=None)[0]
            assert np.max(np.abs(Ak.T @ coef - drop.T)) < 1e-9


def test_reduction_is_greedy_in_canonical_order():
    """The kept set is the greedy basis of the rows in the canonical order
    (cliques N..1, natural order inside a clique): a row is dropped exactly
    when it lies in the span of the rows before it. Checked with an
    orthonormal basis of the kept rows grown by Gram-Schmidt (projected
    twice), independently of the Cholesky used by reduce_rows."""
    for p in (wl.toy_problem(N=3), wl.pendulum_problem(N=2, theta0=0.13)):
        sdp = R.relax(p)
        keep, _ = O.reduce_rows(sdp)
        Ad = sdp.A.toarray()
        Q = np.zeros((int(keep.sum()), Ad.shape[1]))
        k = 0
        for row in O.canonical_row_order(sdp):
            a = Ad[row]
            r = a - Q[:k].T @ (Q[:k] @ a)
            r = r - Q[:k].T @ (Q[:k] @ r)
            resid = np.linalg.norm(r) / np.linalg.norm(a)
            assert (resid < 1e-6) == (not keep[row]), (p.name, row, resid)
            if keep[row]:
                Q[k] = r / np.linalg.norm(r)
                k += 1


def test_ysolver_backward_error():
    p = wl.pendulum_problem(N=4, theta0=0.05)
    red = O.reduce(R.relax(p))
    ys = O.YSolver(red.A)
    r = np.random.default_rng(0).standard_normal(red.m)
    y = ys(r)
    assert np.linalg.norm(red.A @ (red.A.T @ y) - r) <= 1e-12 * np.linalg.norm(r) * 1e2


def _toy_brute(p):
    N = p.N

    def cost(u):
        return p.objective(_toy_rollout(p, np.clip(u, -1, 1)))
    g = np.linspace(-1, 1, 201)
    if N == 2:
        U0, U1 = np.meshgrid(g, g, indexing="ij")
        vals = np.vectorize(lambda a, b: cost([a, b]))(U0, U1)
        i = np.unravel_index(np.argmin(vals), vals.shape)
        u0 = np.array([g[i[0]], g[i[1]]])
    else:
        u0 = np.zeros(N)
        best = np.inf
        for a in np.linspace(-1, 1, 21):
            for b in np.linspace(-1, 1, 21):
                for c in np.linspace(-1, 1, 21):
                    v = cost([a, b, c])
                    if v < best:
                        best, u0 = v, np.array([a, b, c])
    r = so.minimize(cost, u0, bounds=[(-1, 1)] * N, method="L-BFGS-B", options=dict(ftol=1e-15, gtol=1e-12))
    return min(r.fun, cost(u0))


def _pend_brute(p):
    N = p.N

    def cost(U):
        z = _pend_rollout(p, np.clip(U, -1, 1))
        W = z[2::4]
        if np.max(np.abs(W)) > 1.0:
            return np.inf
        return p.objective(z)
    g = np.linspace(-1, 1, 201)
    best, u0 = np.inf, None
    for a in g:
        for b in g:
            v = cost([a, b])
            if v < best:
                best, u0 = v, np.array([a, b])
    r = so.minimize(cost, u0, bounds=[(-1, 1)] * N, method="L-BFGS-B", options=dict(ftol=1e-15, gtol=1e-12))
    return min(r.fun, best)


@pytest.mark.parametrize("case", ["toy2", "toy3", "pend2"])
def test_relaxation_matches_brute_force(case):
    if case.startswith("toy"):
        p = wl.toy_problem(N=int(case[-1]))
        pbf = _toy_brute(p)
    else:
        p = wl.pendulum_problem(N=2, theta0=0.12)
        pbf = _pend_brute(p)
    red = O.reduce(R.relax(p))
    res = O.solve(red, O.Options(tol=1e-9, maxiter=40000))
    assert res.converged
    cert = CE.certify(p, red, res.X, res.y)
    # Theorem 1 (ii): p*_kappa <= p*
    assert res.pobj <= pbf + 1e-6 * (1 + abs(pbf))
    # valid lower bound <= p* and xi >= 0 (eq. valid-lowerbound, eq. suboptimality)
    assert cert.lower_bound <= pbf + 1e-9
    assert cert.xi >= -1e-12
    # Theorem 1 (iii): rank one => tight
    if cert.max_ratio < 1e-5:
        assert abs(res.pobj - pbf) <= 1e-5 * (1 + abs(pbf))
        assert cert.feasible
        assert cert.phat >= pbf - 1e-9 * (1 + abs(pbf))


def test_admm_detects_wrong_sign():
    """A planted mistake (sign of C flipped in Step 2) must break the brute-force pin."""
    p = wl.toy_problem(N=2)
    red = O.reduce(R.relax(p))
    good = O.solve(red, O.Options(tol=1e-8, maxiter=20000))
    bad_sdp = R.relax(p)
    bad_sdp.C = -bad_sdp.C
    bad = O.solve(O.ReducedSDP(bad_sdp, red.keep, red.A, red.b, red.blocks), O.Options(tol=1e-8, maxiter=20000))
    assert abs(bad.pobj - good.pobj) > 1e-2


# --------------------------------------------------------------------------
# closed forms of Algorithm 1 and of the residuals (eq. kkt-residual)
# --------------------------------------------------------------------------
def _trace_sdp(Cmats, seed=0):
    """min <C, X> s.t. tr(X_beta) = 1 for every block, X_beta PSD: the optimum
    of each block is lambda_min(C_beta), attained at v v^T (v its eigenvector),
    and the dual is y_beta = lambda_min(C_beta), S_beta = C_beta - y_beta I."""
    blocks, off, C, rows = [], 0, [], []
    for k, Cm in enumerate(Cmats):
        n = Cm.shape[0]
        blocks.append(R.Block("M", k, -1, n, off))
        C.append(R.svec(Cm))
        rows.append((off, R.svec(np.eye(n))))
        off += n * (n + 1) // 2
    A = np.zeros((len(Cmats), off))
    for i, (o, v) in enumerate(rows):
        A[i, o:o + len(v)] = v
    A = sp.csr_matrix(A)
    sdp = R.SDP(blocks, off, np.concatenate(C), A, np.ones(len(Cmats)), np.zeros(len(Cmats), np.int8),
                np.arange(len(Cmats)), len(Cmats), 0, 2, None)
    return O.ReducedSDP(sdp, np.ones(len(Cmats), bool), A, sdp.b, sdp.block_slices())


def test_algorithm1_reaches_the_closed_form_optimum():
    rng = np.random.default_rng(21)
    mats = []
    for n in (3, 5, 8):
        G = rng.standard_normal((n, n))
        mats.append(0.5 * (G + G.T))
    red = _trace_sdp(mats)
    res = O.solve(red, O.Options(tol=1e-10, maxiter=20000))
    assert res.converged
    want = sum(np.linalg.eigvalsh(M)[0] for M in mats)
    assert abs(res.pobj - want) <= 1e-8 * (1 + abs(want))
    assert abs(res.dobj - want) <= 1e-8 * (1 + abs(want))
    for k, M in enumerate(mats):
        assert abs(res.y[k] - np.linalg.eigvalsh(M)[0]) <= 1e-7
        b = red.blocks[k]
        X = R.smat(res.X[b[0]:b[0] + b[1] * (b[1] + 1) // 2], b[1])
        v = np.linalg.eigh(M)[1][:, 0]
        assert np.max(np.abs(X - np.outer(v, v))) <= 1e-6


def test_residuals_closed_form():
    red = _trace_sdp([np.diag([1.0, -2.0]), np.diag([3.0, 4.0, 5.0])])
    C = red.sdp.C
    zx, zy = np.zeros(red.sdp.nsvec), np.zeros(red.m)
    ep, ed, eg, pobj, dobj = O.residuals(red, C, zx, zy, zx)
    nb, nc = np.linalg.norm(red.b), np.linalg.norm(C)
    assert abs(ep - nb / (1 + nb)) < 1e-15 and abs(ed - nc / (1 + nc)) < 1e-15 and eg == 0.0
    # at the exact primal-dual pair all three vanish
    X = np.concatenate([R.svec(np.diag([0.0, 1.0])), R.svec(np.diag([1.0, 0.0, 0.0]))])
    y = np.array([-2.0, 3.0])
    S = C - red.A.T @ y
    ep, ed, eg, pobj, dobj = O.residuals(red, C, X, y, S)
    assert max(ep, ed, eg) < 1e-15 and pobj == dobj == 1.0


def test_paper_pendulum_relaxation_matches_brute_force():
    """The paper's own pendulum model (variational integrator on SO(2)) at N = 2:
    the relaxation is tight (rank 1) and its optimum equals a brute-force search
    over both controls of the explicit simulation, with f_c >= f_c,min enforced."""
    from test_oracle_relax import _paper_pend_rollout
    p = wl.paper_pendulum_problem(N=2, theta0=0.3, thetadot0=0.7)
    fc_min = p.meta["fc_min"]

    def cost(U):
        U = np.clip(U, -1, 1)
        with np.errstate(invalid="ignore"):
            z = _paper_pend_rollout(p, U)
        fc = np.array([z[5 * k + 2] for k in range(1, p.N + 1)])    # x_k = (r_c, r_s, f_c, f_s) at z[5k:5k+4]
        if not np.all(np.isfinite(z)) or np.any(fc < fc_min):
            return np.inf
        return p.objective(z)
    g = np.linspace(-1, 1, 201)
    best, u0 = np.inf, None
    for a in g:
        for b in g:
            v = cost([a, b])
            if v < best:
                best, u0 = v, np.array([a, b])
    r = so.minimize(cost, u0, bounds=[(-1, 1)] * 2, method="L-BFGS-B", options=dict(ftol=1e-15, gtol=1e-12))
    pbf = min(r.fun, best)
    red = O.reduce(R.relax(p))
    res = O.solve(red, O.Options(tol=1e-9, maxiter=40000))
    cert = CE.certify(p, red, res.X, res.y)
    assert res.converged and cert.rank_one and cert.feasible
    assert res.pobj <= pbf + 1e-6 * (1 + abs(pbf))
    assert abs(res.pobj - pbf) <= 1e-6 * (1 + abs(pbf))
    assert cert.lower_bound <= pbf + 1e-9


def test_sigma_rule_recovers_from_a_badly_scaled_start(monkeypatch):
    """The sigma rule (reading 7: balance eta_d against max(eta_p, eta_g))
    pinned by its effect, not its formula: on the trace-constrained SDP with
    a closed-form optimum, with the cost scaled by 1e-3, 1 or 1e3 and
    sigma0 in {1e-3, 10, 1e3}, Algorithm 1 reaches the closed-form optimum
    within 3,000 iterations every time; the same rule with its two branches
    swapped (a plausible sign mistake, planted here on the CPU) does not."""
    rng = np.random.default_rng(21)
    mats = []
    for n in (3, 5, 8):
        G = rng.standard_normal((n, n))
        mats.append(0.5 * (G + G.T))
    for scale in (1e-3, 1.0, 1e3):
        red = _trace_sdp([scale * M for M in mats])
        want = scale * sum(np.linalg.eigvalsh(M)[0] for M in mats)
        for s0 in (1e-3, 10.0, 1e3):
            res = O.solve(red, O.Options(tol=1e-8, maxiter=3000, sigma0=s0))
            assert res.converged, (scale, s0, res.iters)
            assert abs(res.pobj - want) <= 1e-6 * (1 + abs(want)), (scale, s0)

    def swapped(sigma, eta_p, eta_d, eta_g, opt):
        eta_pg = max(eta_p, eta_g)
        if eta_pg > opt.sigma_ratio * eta_d:
            sigma *= opt.sigma_factor
        elif eta_d > opt.sigma_ratio * eta_pg:
            sigma /= opt.sigma_factor
        return min(max(sigma, opt.sigma_min), opt.sigma_max)

    monkeypatch.setattr(O, "sigma_update", swapped)
    fails = 0
    for scale, s0 in ((1.0, 10.0), (1e3, 10.0), (1e-3, 1e-3)):
        red = _trace_sdp([scale * M for M in mats])
        fails += not O.solve(red, O.Options(tol=1e-8, maxiter=3000, sigma0=s0)).converged
    assert fails == 3
