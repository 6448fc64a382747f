"""Oracle: Algorithm 1 (sGS-ADMM) for the SDP pair (eq. standardsdp, eq. standardsdp-dual).

Everything here is plain FP64 NumPy/SciPy:
  * project_psd      Pi(X_beta) = Q max(0, W) Q^T (Sec. 4, parallel PSD cone
                     projection), with numpy.linalg.eigh as the eigensolver;
  * A_op / At_op     A(X) = (<A_i, X>)_i and A^* y = sum_l y_l A_l (Sec. 3),
                     as scipy sparse products in svec coordinates;
  * reduce_rows      removal of linearly dependent rows so that A A^* > 0,
                     decided by a pivot-skipping Cholesky in a fixed order
                     (cliques N..1, natural row order inside a clique), on
                     the Gram matrix of the rows other than A_mom after
                     projecting out span(A_mom) (other_rows_gram);
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
import scipy.sparse.csgraph  # noqa: F401  (sp.csgraph)
import scipy.sparse.linalg as spla

from .relax import KIND_CONS, KIND_MOM, SDP, smat, svec

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


def other_rows_gram(sdp: SDP):
    """Gram matrix of the rows other than A_mom after projecting out span(A_mom).

    With A_s the A_mom rows and A_o the others, the projection of A_o on the
    orthogonal complement of the row space of A_s has the Gram matrix
        S = A_o A_o^T - (A_s A_o^T)^T (A_s A_s^T)^{-1} (A_s A_o^T),
    formed here with sparse products and a sparse solve (A_s A_s^T is block
    diagonal: one block per monomial with duplicate entries). Returns S
    (sparse, rows and columns in the natural order of the other rows) and
    the row ids of those rows.
    """
    A = sdp.A.tocsr()
    is_s = sdp.row_kind == KIND_MOM
    As, Ao = A[is_s], A[~is_s]
    other_rows = np.nonzero(~is_s)[0]
    if As.shape[0] == 0:
        return (Ao @ Ao.T).tocsr(), other_rows
    Gs = (As @ As.T).tocsr()
    B = (As @ Ao.T).tocsc()
    S = (Ao @ Ao.T) - (B.T @ block_diagonal_inverse(Gs) @ B)
    return sp.csr_matrix(S), other_rows


def block_diagonal_inverse(G: sp.csr_matrix) -> sp.csr_matrix:
    """Inverse of a symmetric positive definite block-diagonal sparse matrix
    whose blocks are small (the connected components of its graph), each
    block inverted densely."""
    ncomp, lab = sp.csgraph.connected_components(G, directed=False)
    order = np.argsort(lab, kind="stable")
    bounds = np.searchsorted(lab[order], np.arange(ncomp + 1))
    rows, cols, vals = [], [], []
    for c in range(ncomp):
        ids = order[bounds[c]:bounds[c + 1]]
        inv = np.linalg.inv(G[ids][:, ids].toarray())
        rows.append(np.repeat(ids, len(ids)))
        cols.append(np.tile(ids, len(ids)))
        vals.append(inv.ravel())
    n = G.shape[0]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def reduce_rows(sdp: SDP, tol: float = RANK_TOL):
    """Boolean keep-mask over the rows of A and the relative pivots.

    A row is dropped iff its Cholesky pivot in the canonical order (its
    squared distance to the span of the kept rows before it) is at most
    tol times its squared norm. Moment-duplication rows (A_mom) each own an
    entry no other row touches, so they are always independent; and a row of
    clique k shares no entry with the A_mom rows of any other clique.
    Hence the test may run on the other rows after projecting out the span
    of all A_mom rows (Gram matrix S of other_rows_gram).

    The pivot-skipping Cholesky of S runs in the canonical order (cliques
    N..1, natural row order inside a clique). In that order S is block
    tridiagonal: the rows of clique k meet only each other and the consensus
    rows of clique k-1 (the one kind of row of clique k-1 that touches M_k).
    So the elimination of clique k's rows is carried out on a dense window
    holding those rows and the consensus rows of clique k-1; what it
    subtracts from the consensus rows' Gram is carried to clique k-1's
    window. This is the same scalar algorithm on the same matrix, entry by
    entry, without storing the zero blocks.
    """
    S, other_rows = other_rows_gram(sdp)
    S = S.tocsr()
    rc = sdp.row_clique[other_rows]
    rk = sdp.row_kind[other_rows]
    keep_o = np.zeros(len(other_rows), dtype=bool)
    rel_o = np.zeros(len(other_rows))
    carry = None          # Schur update waiting for the consensus rows of the clique below
    for k in range(sdp.N - 1, -1, -1):
        G = np.nonzero(rc == k)[0]                                   # natural order
        P = np.nonzero((rc == k - 1) & (rk == KIND_CONS))[0] if k > 0 else np.zeros(0, int)
        idx = np.concatenate([G, P])
        W = S[idx][:, idx].toarray()
        nG = len(G)
        W[nG:, nG:] = 0.0                      # the consensus rows' own Gram enters in their window
        if carry is not None:
            cons = np.nonzero(rk[G] == KIND_CONS)[0]
            W[np.ix_(cons, cons)] -= carry
        d0 = np.array(S[G, G]).ravel()         # squared norms of the projected rows
        for j in range(nG):
            d = W[j, j]
            rel_o[G[j]] = d / d0[j] if d0[j] > 0 else 0.0
            if d0[j] <= 0 or d <= tol * d0[j]:
                W[j, j + 1:] = 0.0
                W[j + 1:, j] = 0.0
                continue
            keep_o[G[j]] = True
            l = W[j + 1:, j] / np.sqrt(d)
            nz = np.nonzero(l)[0]
            if len(nz):
                lo, hi = nz[0], nz[-1] + 1
                if 2 * len(nz) >= hi - lo:      # dense enough: update the whole range (zeros change nothing)
                    W[j + 1 + lo:j + 1 + hi, j + 1 + lo:j + 1 + hi] -= np.outer(l[lo:hi], l[lo:hi])
                else:
                    sub = j + 1 + nz
                    W[np.ix_(sub, sub)] -= np.outer(l[nz], l[nz])
        carry = -W[nG:, nG:] if len(P) else None
    keep = sdp.row_kind == KIND_MOM
    keep = keep.copy()
    keep[other_rows[keep_o]] = True
    rel_full = np.ones(sdp.m)
    rel_full[other_rows] = rel_o
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
