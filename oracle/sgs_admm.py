"""Oracle: Algorithm 1 (sGS-ADMM) for the SDP pair (eq. standardsdp, eq. standardsdp-dual).

Everything here is plain FP64 NumPy/SciPy:
  * project_psd      Pi(X_beta) = Q max(0, W) Q^T (Sec. 4, parallel PSD cone
                     projection), with numpy.linalg.eigh as the eigensolver;
  * A_op / At_op     A(X) = (<A_i, X>)_i and A^* y = sum_l y_l A_l (Sec. 3),
                     as scipy sparse products in svec coordinates;
  * reduce_rows      removal of linearly dependent rows so that A A^* > 0,
                     decided by a pivot-skipping Cholesky in a fixed order
                     (cliques N..1, natural row order inside a clique);
  * YSolver          y = (A A^*)^{-1} r with a sparse LU of A A^* (library);
  * solve            Steps 1-4 of Algorithm 1 and the terminal conditions
                     of eq. (kkt-residual).

Readings of the paper that are ours (the paper leaves them open): the
penalty sigma is adapted every 20 iterations by halving it when
max(eta_p, eta_g) > 5 eta_d and doubling it when eta_d > 5 max(eta_p, eta_g)
(clipped to [1e-4, 1e4]);
tau = 1.618; sigma0 = 10; X0 = S0 = 0; residuals use (X^{k+1}, y^{k+1}, S^{k+1}) and the
row-reduced A.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .relax import KIND_MOM, SDP, smat, svec

RANK_TOL = 1e-8


# --------------------------------------------------------------------------
# PSD projection (Sec. 4)
# --------------------------------------------------------------------------
def project_block(M: np.ndarray) -> np.ndarray:
    """Pi_{S+}(M) = Q max(0, W) Q^T from the eigendecomposition M = Q W Q^T."""
    W, Q = np.linalg.eigh(0.5 * (M + M.T))
    return (Q * np.maximum(W, 0.0)) @ Q.T


def project_psd(x: np.ndarray, blocks) -> np.ndarray:
    """Apply Pi to every block of an svec vector; blocks = [(offset, n), ...]."""
    out = np.empty_like(x)
    for off, n in blocks:
        t = n * (n + 1) // 2
        out[off:off + t] = svec(project_block(smat(x[off:off + t], n)))
    return out


def min_eig_blocks(x: np.ndarray, blocks) -> np.ndarray:
    return np.array([np.linalg.eigvalsh(smat(x[off:off + n * (n + 1) // 2], n))[0]
                     for off, n in blocks])


# --------------------------------------------------------------------------
# linear maps (Sec. 3)
# --------------------------------------------------------------------------
def A_op(A: sp.csr_matrix, x: np.ndarray) -> np.ndarray:
    return A @ x


def At_op(A: sp.csr_matrix, y: np.ndarray) -> np.ndarray:
    return A.T @ y


# --------------------------------------------------------------------------
# row reduction: keep a row iff it is not in the span of the rows before it
# --------------------------------------------------------------------------
def canonical_row_order(sdp: SDP) -> np.ndarray:
    """Cliques N..1; inside a clique rows keep their natural order."""
    idx = np.arange(sdp.m)
    return np.concatenate([idx[sdp.row_clique == k] for k in range(sdp.N - 1, -1, -1)])


def reduce_rows(sdp: SDP, tol: float = RANK_TOL):
    """Boolean keep-mask over the rows of A and the relative pivots.

    A row is dropped iff its Cholesky pivot in the canonical order (its
    squared distance to the span of the kept rows before it) is at most
    tol times its squared norm. Moment-duplication rows (A_mom) each own an
    entry no other row touches, so they are always independent; and a row of
    clique k shares no entry with the A_mom rows of any other clique.
    Hence the test may run on the other rows after projecting out the span
    of all A_mom rows, which is what is done here.
    """
    A = sdp.A.tocsr()
    is_s = sdp.row_kind == KIND_MOM
    As, Ao = A[is_s], A[~is_s]
    Gs = (As @ As.T).tocsc()
    lu = spla.splu(Gs)
    Z = lu.solve((As @ Ao.T).toarray())             # (As As^T)^{-1} As Ao^T
    Ahat = Ao.toarray() - (As.T @ Z).T              # Ao minus its projection on span(As)
    other_rows = np.nonzero(~is_s)[0]
    order_all = canonical_row_order(sdp)
    pos = {r: i for i, r in enumerate(other_rows)}
    order = np.array([pos[r] for r in order_all if not is_s[r]])
    G = Ahat[order] @ Ahat[order].T
    m = len(order)
    keep_o = np.zeros(m, dtype=bool)
    rel = np.zeros(m)
    for i in range(m):
        d = G[i, i]
        nrm = np.dot(Ahat[order[i]], Ahat[order[i]])
        rel[i] = d / nrm if nrm > 0 else 0.0
        if nrm <= 0 or d <= tol * nrm:
            G[i, i + 1:] = 0.0
            G[i + 1:, i] = 0.0
            continue
        keep_o[i] = True
        l = G[i + 1:, i] / np.sqrt(d)
        nz = np.nonzero(l)[0]
        if len(nz):
            sub = i + 1 + nz
            G[np.ix_(sub, sub)] -= np.outer(l[nz], l[nz])
    keep = is_s.copy()
    keep[other_rows[order[keep_o]]] = True
    rel_full = np.ones(sdp.m)
    rel_full[other_rows[order]] = rel
    return keep, rel_full


@dataclass
class ReducedSDP:
    sdp: SDP
    keep: np.ndarray
    A: sp.csr_matrix
    b: np.ndarray
    blocks: list = field(default_factory=list)

    @property
    def m(self):
        return self.A.shape[0]


def reduce(sdp: SDP, tol: float = RANK_TOL) -> ReducedSDP:
    keep, _ = reduce_rows(sdp, tol)
    return ReducedSDP(sdp, keep, sdp.A[keep].tocsr(), sdp.b[keep], sdp.block_slices())


class YSolver:
    """y = (A A^T)^{-1} r for the row-reduced A (sparse LU as a library step)."""

    def __init__(self, A: sp.csr_matrix):
        self.lu = spla.splu((A @ A.T).tocsc())

    def __call__(self, r):
        return self.lu.solve(r)


# --------------------------------------------------------------------------
# Algorithm 1
# --------------------------------------------------------------------------
@dataclass
class Options:
    tol: float = 1e-6
    maxiter: int = 50000
    sigma0: float = 10.0
    tau: float = 1.618
    sigma_every: int = 20
    sigma_ratio: float = 5.0
    sigma_factor: float = 2.0
    sigma_min: float = 1e-4
    sigma_max: float = 1e4


@dataclass
class Result:
    X: np.ndarray
    y: np.ndarray
    S: np.ndarray
    iters: int
    pobj: float
    dobj: float
    eta_p: float
    eta_d: float
    eta_g: float
    sigma: float
    converged: bool
    history: list


def residuals(red: ReducedSDP, C, X, y, S, Aty=None):
    """eta_p, eta_d, eta_g of eq. (kkt-residual); norms are svec 2-norms."""
    A, b = red.A, red.b
    if Aty is None:
        Aty = A.T @ y
    eta_p = np.linalg.norm(A @ X - b) / (1.0 + np.linalg.norm(b))
    eta_d = np.linalg.norm(Aty + S - C) / (1.0 + np.linalg.norm(C))
    pobj, dobj = float(C @ X), float(b @ y)
    eta_g = abs(pobj - dobj) / (1.0 + abs(pobj) + abs(dobj))
    return eta_p, eta_d, eta_g, pobj, dobj


def sigma_update(sigma, eta_p, eta_d, eta_g, opt: Options):
    """Balance the dual residual against the primal one (eta_p and the gap eta_g)."""
    eta_pg = max(eta_p, eta_g)
    if eta_pg > opt.sigma_ratio * eta_d:
        sigma /= opt.sigma_factor
    elif eta_d > opt.sigma_ratio * eta_pg:
        sigma *= opt.sigma_factor
    return min(max(sigma, opt.sigma_min), opt.sigma_max)


def solve(red: ReducedSDP, opt: Options = Options(), X0=None, S0=None, sigma=None,
          ysolver: YSolver | None = None, record_every: int = 0) -> Result:
    """sGS-ADMM (Algorithm 1) from (X0, S0); stops when max(eta) <= tol or at maxiter."""
    C = red.sdp.C
    A, b = red.A, red.b
    At = A.T.tocsr()
    blocks = red.blocks
    X = np.zeros(red.sdp.nsvec) if X0 is None else X0.copy()
    S = np.zeros(red.sdp.nsvec) if S0 is None else S0.copy()
    sigma = opt.sigma0 if sigma is None else sigma
    ys = ysolver or YSolver(A)
    y = np.zeros(red.m)
    hist = []
    it = 0
    converged = False
    eta = (np.inf,) * 3
    pobj = dobj = 0.0
    while it < opt.maxiter:
        # Step 1
        r = b / sigma - A @ (X / sigma + S - C)
        yh = ys(r)
        # Step 2
        Xb = X + sigma * (At @ yh - C)
        S = (project_psd(Xb, blocks) - Xb) / sigma
        # Step 3
        r = b / sigma - A @ (X / sigma + S - C)
        y = ys(r)
        # Step 4
        Aty = At @ y
        X = X + opt.tau * sigma * (S + Aty - C)
        it += 1
        ep, ed, eg, pobj, dobj = residuals(red, C, X, y, S, Aty)
        eta = (ep, ed, eg)
        if record_every and it % record_every == 0:
            hist.append((it, ep, ed, eg, sigma, pobj, dobj))
        if max(eta) <= opt.tol:
            converged = True
            break
        if it % opt.sigma_every == 0:
            sigma = sigma_update(sigma, ep, ed, eg, opt)
    return Result(X, y, S, it, pobj, dobj, eta[0], eta[1], eta[2], sigma, converged, hist)
