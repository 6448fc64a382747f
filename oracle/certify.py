"""Oracle: rank-1 test, solution extraction and the suboptimality certificate.

* Theorem 1 (iii): rank M_k = 1 for all k certifies tightness; the ratio
  lambda_2 / lambda_1 of each moment block is reported.
* Extraction heuristic (Sec. 2.2): top eigenvector v_k of M_k, normalised
  by its first entry; its degree-1 entries give z_bar(I_k).
* Local step: the paper runs fmincon from z_bar. Here the controls of z_bar
  are clipped to the variable box and the equalities of each clique are
  solved for its new state by Gauss-Newton, clique by clique (a rollout).
* Valid lower bound (eq. valid-lowerbound) with R_beta of the theorem in
  App. C, and the refined gap xi (eq. suboptimality-gap).

R_beta reading: trace(M_k(z)) = ||[z]_kappa||^2 <= s(n, kappa) max(1, R)^(2 kappa)
(the printed proof drops the power) and, for localizing blocks,
g <= sum_t |c_t| max(1, R)^(deg t) over the box, which bounds the printed
max g from above and keeps the lower bound valid.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .relax import SDP, _deg, _poly_terms, s_count, smat


def r_beta(problem, sdp: SDP) -> np.ndarray:
    R = max(1.0, float(problem.R))
    out = []
    for blk in sdp.blocks:
        if blk.kind == "M":
            out.append(s_count(sdp.nv, sdp.kappa) * R ** (2 * sdp.kappa))
        else:
            gt = _poly_terms(problem.cliques[blk.clique].g[blk.index])
            dg = math.ceil(_deg(gt) / 2)
            gmax = sum(abs(c) * R ** sum(e) for c, e in gt)
            out.append(gmax * s_count(sdp.nv, sdp.kappa - dg) * R ** (2 * (sdp.kappa - dg)))
    return np.array(out)


def _eval(terms, z):
    return sum(c * np.prod(z ** np.array(e, dtype=np.float64)) for c, e in terms)


def _grad(terms, z, idx):
    """d/dz_i of the polynomial for each i in idx."""
    g = np.zeros(len(idx))
    for c, e in terms:
        e = np.array(e, dtype=np.float64)
        for t, i in enumerate(idx):
            if e[i] == 0:
                continue
            ee = e.copy()
            ee[i] -= 1
            g[t] += c * e[i] * np.prod(z ** ee)
    return g


def extract(problem, sdp: SDP, X: np.ndarray):
    """Per clique (lambda_2/lambda_1, z_bar(I_k)); z_bar assembled into a global vector."""
    nv, dx, du = problem.nv, problem.dx, problem.du
    ratios, zbar = [], np.zeros(problem.nz)
    for blk in sdp.blocks:
        if blk.kind != "M":
            continue
        M = smat(X[blk.offset: blk.offset + blk.n * (blk.n + 1) // 2], blk.n)
        W, Q = np.linalg.eigh(M)
        ratios.append(W[-2] / W[-1] if W[-1] > 0 else np.inf)
        v = Q[:, -1] / Q[0, -1]
        zk = v[1:1 + nv]
        k = blk.clique
        s = k * (dx + du)
        zbar[s: s + dx + du] = zk[: dx + du]
        if k == problem.N - 1:
            zbar[s + dx + du: s + nv] = zk[dx + du:]
    return np.array(ratios), zbar


def rollout(problem, zbar, iters: int = 60):
    """Clip controls to [-R, R] and solve each clique's equalities for its new state."""
    dx, du, nv = problem.dx, problem.du, problem.nv
    z = zbar.copy()
    R = problem.R
    for k in range(problem.N):
        s = k * (dx + du)
        z[s + dx: s + dx + du] = np.clip(z[s + dx: s + dx + du], -R, R)
        unknown = list(range(dx + du, nv)) if k > 0 else list(range(dx)) + list(range(dx + du, nv))
        hs = [_poly_terms(h) for h in problem.cliques[k].h]
        zk = z[s: s + nv].copy()
        for _ in range(iters):
            F = np.array([_eval(t, zk) for t in hs])
            if np.max(np.abs(F)) < 1e-14:
                break
            J = np.array([_grad(t, zk, unknown) for t in hs])
            step = np.linalg.lstsq(J, -F, rcond=None)[0]
            zk[unknown] += step
        z[s: s + nv] = zk
    return z


def feasibility(problem, z):
    """(max |h|, min g) over all cliques at the global point z."""
    hmax, gmin = 0.0, np.inf
    for k, c in enumerate(problem.cliques):
        zk = problem.clique_vars(z, k)
        for h in c.h:
            hmax = max(hmax, abs(_eval(_poly_terms(h), zk)))
        for g in c.g:
            gmin = min(gmin, _eval(_poly_terms(g), zk))
    return hmax, gmin


@dataclass
class Certificate:
    ratios: np.ndarray
    max_ratio: float
    zbar: np.ndarray
    zhat: np.ndarray
    hmax: float
    gmin: float
    feasible: bool
    phat: float
    lower_bound: float
    xi: float
    rank_one: bool
    certified: bool


def certify(problem, red, X, y, rank_tol=1e-4, xi_tol=1e-2, feas_tol=1e-9) -> Certificate:
    sdp = red.sdp
    ratios, zbar = extract(problem, sdp, X)
    zhat = rollout(problem, zbar)
    hmax, gmin = feasibility(problem, zhat)
    feasible = hmax <= feas_tol and gmin >= -feas_tol
    phat = problem.objective(zhat)
    Z = sdp.C - red.A.T @ y
    lmin = np.array([np.linalg.eigvalsh(smat(Z[b.offset: b.offset + b.n * (b.n + 1) // 2], b.n))[0]
                     for b in sdp.blocks])
    lb = float(red.b @ y + np.sum(r_beta(problem, sdp) * np.minimum(0.0, lmin)))
    xi = (phat - lb) / (1.0 + abs(phat) + abs(lb))
    mr = float(np.max(ratios))
    rank_one = mr <= rank_tol
    return Certificate(ratios, mr, zbar, zhat, hmax, gmin, feasible, phat, lb, xi, rank_one,
                       bool(rank_one and feasible and xi <= xi_tol))


# --------------------------------------------------------------------------
# flat extension and partial rank-1 tests of one moment matrix (Sec. 2.2:
# the flat-extension condition generalises rank 1; App. car back-in: the
# submatrix of the trajectory variables can be rank-1 when M_k is not)
# --------------------------------------------------------------------------
def _numerical_rank(W, tol):
    top = max(W[-1], 0.0)
    return int(np.sum(W > tol * top)) if top > 0 else 0


def moment_rank_tests(M, nv: int, vars_mask=None, tol: float = 1e-8):
    """Rank tests of a moment matrix M of order 2 in nv variables (basis [z]_2,
    graded lexicographic order).

    rank      numerical rank of M (eigenvalues above tol * lambda_max)
    rank_low  the same for the principal submatrix on [z]_1 (degree <= 1)
    flat      rank == rank_low (flat extension: the moments come from a
              measure with exactly rank atoms)
    ratio_sub lambda_2 / lambda_1 of the principal submatrix on the monomials
              whose variables all lie in vars_mask (all variables if None)
    zbar_sub  its top eigenvector scaled to a leading 1, entries of the
              degree-1 monomials of the selected variables (NaN elsewhere)
    """
    from .relax import monomial_basis
    basis = monomial_basis(nv, 2)
    M = np.asarray(M, dtype=np.float64)
    sel = np.ones(nv, bool) if vars_mask is None else np.asarray(vars_mask, bool)
    W = np.linalg.eigvalsh(M)
    low = [i for i, e in enumerate(basis) if sum(e) <= 1]
    W_low = np.linalg.eigvalsh(M[np.ix_(low, low)])
    sub = [i for i, e in enumerate(basis) if all(sel[t] or e[t] == 0 for t in range(nv))]
    Ws, Qs = np.linalg.eigh(M[np.ix_(sub, sub)])
    ratio = Ws[-2] / Ws[-1] if (len(sub) > 1 and Ws[-1] > 0) else (0.0 if Ws[-1] > 0 else np.inf)
    v = Qs[:, -1] / Qs[0, -1]
    zbar = np.full(nv, np.nan)
    for j, i in enumerate(sub):
        e = basis[i]
        if sum(e) == 1:
            zbar[e.index(1)] = v[j]
    rank, rank_low = _numerical_rank(W, tol), _numerical_rank(W_low, tol)
    return dict(n=len(basis), rank=rank, rank_low=rank_low, flat=rank == rank_low, n_sub=len(sub),
                ratio_sub=float(ratio), lambda_max=float(W[-1]), zbar_sub=zbar)
