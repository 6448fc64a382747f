"""Oracle: sparse moment relaxation -> standard multi-block SDP (FP64, plain Python).

Follows Prop. 1 (sparse moment relaxation, order kappa) and the PSD-only
conversion of Sec. 2.3 (eq. standardsdp): X is the tuple of all moment
matrices M_k and localizing matrices L_{k,i} (eq. def-X), C encodes the
objective and A(X) = b stacks four kinds of linear constraints
(A_mom, A_ineq, A_eq, A_sen of Sec. 2.3) plus the normalisation phi_0 = 1.

Conventions (readings of the paper, all checked against the worked example
of Sec. 2.3 by tests):
  * monomial basis [z]_d: graded, lexicographic in clique variable order
    within each degree (the printed basis of eq. toy-M2);
  * a monomial alpha of M_k is represented by its first occurrence in
    column-major upper-triangular order; this reproduces every index the
    paper prints (M2(4,6), M2(3,3), M2(3,6), M2(2,3), M2(1,4), M3(2,5) ...);
  * svec is the SDPT3 vectorisation: column-major upper triangle with the
    off-diagonal entries times sqrt(2), so <A, B> = svec(A) . svec(B);
  * blocks are ordered M_1, L_{1,1..}, M_2, L_{2,..}, ... and rows by clique;
    inside clique k: A_mom, A_ineq, A_eq, phi_0 row M_k(1,1) = 1, then the
    consensus rows shared with clique k+1 (monomials of degree 1..2 kappa in
    the overlap variables).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

SQRT2 = math.sqrt(2.0)

KIND_MOM, KIND_INEQ, KIND_EQ, KIND_PHI0, KIND_CONS = 0, 1, 2, 3, 4


def s_count(n: int, d: int) -> int:
    """s(n, d) = C(n + d, d), the number of monomials of degree <= d in n variables."""
    return math.comb(n + d, d)


def monomial_basis(nv: int, d: int):
    """[z]_d as exponent tuples: graded, lexicographic in variable order within a degree."""
    out = []
    for deg in range(d + 1):
        for comb in itertools.combinations_with_replacement(range(nv), deg):
            e = [0] * nv
            for i in comb:
                e[i] += 1
            out.append(tuple(e))
    return out


def svec_index(i: int, j: int) -> int:
    """0-based position of entry (i, j), i <= j, in column-major upper svec."""
    if i > j:
        i, j = j, i
    return j * (j + 1) // 2 + i


def svec_scale(i: int, j: int) -> float:
    """Coefficient s with M(i,j) = s * svec(M)[p]: 1 on the diagonal, 1/sqrt(2) off it."""
    return 1.0 if i == j else 1.0 / SQRT2


def upper_entries(n: int):
    """(i, j) pairs in column-major upper-triangular order."""
    return [(i, j) for j in range(n) for i in range(j + 1)]


def _add(e1, e2):
    return tuple(a + b for a, b in zip(e1, e2))


class MomentIndex:
    """Monomial table of one moment matrix ell([z]_kappa [z]_kappa^T)."""

    def __init__(self, nv: int, kappa: int):
        self.basis = monomial_basis(nv, kappa)
        self.n = len(self.basis)
        self.rep = {}          # monomial -> (i, j) first occurrence, column-major upper
        self.entries = {}      # monomial -> list of (i, j) in column-major upper order
        for (i, j) in upper_entries(self.n):
            a = _add(self.basis[i], self.basis[j])
            self.entries.setdefault(a, []).append((i, j))
            if a not in self.rep:
                self.rep[a] = (i, j)


@dataclass
class Block:
    kind: str          # "M" or "L"
    clique: int        # 0-based clique index
    index: int         # localizing index i (0-based), -1 for M
    n: int             # matrix size
    offset: int        # svec offset in X


@dataclass
class SDP:
    blocks: list
    nsvec: int
    C: np.ndarray
    A: sp.csr_matrix
    b: np.ndarray
    row_kind: np.ndarray
    row_clique: np.ndarray
    N: int
    nv: int
    kappa: int
    mindex: MomentIndex

    @property
    def m(self) -> int:
        return self.A.shape[0]

    def block_slices(self):
        return [(blk.offset, blk.n) for blk in self.blocks]


def _poly_terms(poly):
    """Accept a workloads.Poly or a (coef, expo) pair; yield (coef, exponent tuple)."""
    if hasattr(poly, "terms"):
        return [(v, tuple(int(x) for x in k)) for k, v in sorted(poly.terms.items())]
    coef, expo = poly
    return [(float(c), tuple(int(x) for x in e)) for c, e in zip(coef, expo)]


def _deg(terms):
    return max((sum(e) for _, e in terms), default=0)


def relax(problem) -> SDP:
    """Build {C, A, b} of the order-kappa sparse moment relaxation (Prop. 1, Sec. 2.3)."""
    N, nv, kappa, dx = problem.N, problem.nv, problem.kappa, problem.dx
    mi = MomentIndex(nv, kappa)
    nM = mi.n
    # block layout --------------------------------------------------------
    blocks, off = [], 0
    loc_info = []      # per clique: list of (block, basis, g terms)
    for k in range(N):
        blocks.append(Block("M", k, -1, nM, off))
        off += nM * (nM + 1) // 2
        cl = problem.cliques[k]
        lst = []
        for i, g in enumerate(cl.g):
            gt = _poly_terms(g)
            dg = math.ceil(_deg(gt) / 2)
            lb = monomial_basis(nv, kappa - dg)
            blk = Block("L", k, i, len(lb), off)
            off += blk.n * (blk.n + 1) // 2
            blocks.append(blk)
            lst.append((blk, lb, gt))
        loc_info.append(lst)
    nsvec = off
    Mblk = [b for b in blocks if b.kind == "M"]

    def mpos(k, alpha):
        """(global svec index, scale) of the representative entry of alpha in M_k."""
        i, j = mi.rep[alpha]
        return Mblk[k].offset + svec_index(i, j), svec_scale(i, j)

    rows_i, rows_j, rows_v = [], [], []
    b, kinds, cliques = [], [], []

    def emit(entries, rhs, kind, k):
        acc = {}
        for (p, v) in entries:
            acc[p] = acc.get(p, 0.0) + v
        r = len(b)
        for p in sorted(acc):
            if acc[p] != 0.0:
                rows_i.append(r)
                rows_j.append(p)
                rows_v.append(acc[p])
        b.append(rhs)
        kinds.append(kind)
        cliques.append(k)

    C = np.zeros(nsvec)
    for k in range(N):
        cl = problem.cliques[k]
        Mo = Mblk[k].offset
        # objective <C_k, M_k> = ell(f_k) (Sec. 2.3, linear objective)
        for c, e in _poly_terms(cl.f):
            p, s = mpos(k, e)
            C[p] += c * s
        # A_mom: every duplicate entry equals the representative entry
        for (i, j) in upper_entries(nM):
            a = _add(mi.basis[i], mi.basis[j])
            if mi.rep[a] == (i, j):
                continue
            p, s = mpos(k, a)
            emit([(Mo + svec_index(i, j), svec_scale(i, j)), (p, -s)], 0.0, KIND_MOM, k)
        # A_ineq: L_{k,i}(a,b) = ell(g * z^a z^b) as a combination of M_k entries
        for (blk, lb, gt) in loc_info[k]:
            for (a_, b_) in upper_entries(blk.n):
                ent = [(blk.offset + svec_index(a_, b_), svec_scale(a_, b_))]
                mab = _add(lb[a_], lb[b_])
                for c, e in gt:
                    p, s = mpos(k, _add(e, mab))
                    ent.append((p, -c * s))
                emit(ent, 0.0, KIND_INEQ, k)
        # A_eq: ell(h * [z]_{2 kappa - deg h}) = 0 (eq. sparse-momentrelax-equality)
        for h in cl.h:
            ht = _poly_terms(h)
            for mono in monomial_basis(nv, 2 * kappa - _deg(ht)):
                ent = []
                for c, e in ht:
                    p, s = mpos(k, _add(e, mono))
                    ent.append((p, c * s))
                emit(ent, 0.0, KIND_EQ, k)
        # phi_0 = 1 (eq. sparse-momentrelax-normalize), one per clique
        emit([(Mo + svec_index(0, 0), 1.0)], 1.0, KIND_PHI0, k)
        # A_sen: moments of the overlap variables x_k agree in M_k and M_{k+1}
        if k + 1 < N:
            for ov in monomial_basis(dx, 2 * kappa)[1:]:
                ek = (0,) * (nv - dx) + ov
                ek1 = ov + (0,) * (nv - dx)
                p1, s1 = mpos(k, ek)
                p2, s2 = mpos(k + 1, ek1)
                emit([(p1, s1), (p2, -s2)], 0.0, KIND_CONS, k)
    m = len(b)
    A = sp.csr_matrix((rows_v, (rows_i, rows_j)), shape=(m, nsvec))
    A.sum_duplicates()
    A.sort_indices()
    return SDP(blocks, nsvec, C, A, np.array(b), np.array(kinds, dtype=np.int8),
               np.array(cliques, dtype=np.int32), N, nv, kappa, mi)


def svec(M: np.ndarray) -> np.ndarray:
    n = M.shape[0]
    return np.array([M[i, j] * (1.0 if i == j else SQRT2) for (i, j) in upper_entries(n)])


def smat(v: np.ndarray, n: int) -> np.ndarray:
    M = np.zeros((n, n))
    for p, (i, j) in enumerate(upper_entries(n)):
        x = v[p] * (1.0 if i == j else 1.0 / SQRT2)
        M[i, j] = x
        M[j, i] = x
    return M


def lift_rank1(problem, sdp: SDP, z) -> np.ndarray:
    """X(z) of eq. rank1-lifting: M_k = [z]_k [z]_k^T and L_{k,i} = g_{k,i} [z] [z]^T."""
    X = np.zeros(sdp.nsvec)
    for blk in sdp.blocks:
        zk = problem.clique_vars(z, blk.clique)
        if blk.kind == "M":
            basis = sdp.mindex.basis
            g = 1.0
        else:
            gp = problem.cliques[blk.clique].g[blk.index]
            gt = _poly_terms(gp)
            dg = math.ceil(_deg(gt) / 2)
            basis = monomial_basis(sdp.nv, sdp.kappa - dg)
            g = sum(c * np.prod(zk ** np.array(e)) for c, e in gt)
        v = np.array([np.prod(zk ** np.array(e)) for e in basis])
        X[blk.offset: blk.offset + blk.n * (blk.n + 1) // 2] = svec(g * np.outer(v, v))
    return X
