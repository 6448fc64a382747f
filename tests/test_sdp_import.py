"""strom_sdp_import: an SDP given by arrays reproduces the builder's SDP and
the data its y-solve derives (star elimination, Gram weights); malformed
input is rejected with the rule it breaks (CPU, no GPU needed)."""
import numpy as np
import pytest

import workloads as wl
from oracle import relax as OR
from oracle import sgs_admm as OA


@pytest.fixture(scope="module")
def S():
    from paper_2406_05846_gb300 import build
    build.build()
    import paper_2406_05846_gb300 as pkg
    pkg.lib()
    return pkg


PROBLEMS = {
    "toy": lambda: wl.toy_problem(N=3),
    "pendulum": lambda: wl.pendulum_problem(N=5, theta0=0.13, omega0=0.3),
    "pendulum_N1": lambda: wl.pendulum_problem(N=1, theta0=-0.05),
    "cartpole": lambda: wl.cartpole_problem(N=2, x0=0.2, theta0=0.1),
    "rigid": lambda: wl.rigid_body_problem(N=2, disks=[(0.5, -0.3, 0.4), (-1.0, 1.0, 0.6)]),
}


def _import(S, p, a, **over):
    kw = dict(N_=p.N, dx=p.dx, du=p.du, block_n=a.block_n, block_kind=a.block_kind, block_clique=a.block_clique,
              C_=a.C, rowptr=a.rowptr, col=a.col, val=a.val, b=a.b, row_kind=a.row_kind, row_clique=a.row_clique)
    kw.update(over)
    return S.Sdp.from_arrays(**kw)


def _same(x, y):
    return all(np.array_equal(getattr(x, f), getattr(y, f)) for f in x.__dataclass_fields__)


@pytest.mark.parametrize("which", sorted(PROBLEMS))
def test_round_trip_reproduces_builder(S, which):
    p = PROBLEMS[which]()
    built = S.Problem(p).relax()
    a = built.export()
    im = _import(S, p, a)
    assert _same(im.export(), a)
    assert _same(im.star_data(), built.star_data())


@pytest.mark.parametrize("which", ["toy", "pendulum", "rigid"])
def test_oracle_sdp_imports_to_the_builders_structure(S, which):
    p = PROBLEMS[which]()
    o = OR.relax(p)
    im = S.Sdp.from_arrays(p.N, p.dx, p.du, [b.n for b in o.blocks], [0 if b.kind == "M" else 1 for b in o.blocks],
                           [b.clique for b in o.blocks], o.C, o.A.indptr, o.A.indices, o.A.data, o.b, o.row_kind,
                           o.row_clique, block_index=[b.index for b in o.blocks])
    built = S.Problem(p).relax()
    e = im.export()
    assert np.array_equal(e.block_off, [b.offset for b in o.blocks])
    assert np.array_equal(e.val, o.A.data) and np.array_equal(e.C, o.C)
    assert _same(im.star_data(), built.star_data())


def test_star_data_closed_form(S):
    # every moment entry is a representative (weight 1 / (occurrences s_r^2))
    # or a duplicate (weight 0); localizing entries weigh 1; the A_mom rows of
    # a class are exactly the rows whose representative it is
    p = wl.pendulum_problem(N=2)
    sd = S.Problem(p).relax()
    a, st = sd.export(), sd.star_data()
    nM = int(a.block_n[0])
    for k in np.nonzero(a.block_kind == 1)[0]:
        n = int(a.block_n[k])
        assert np.all(st.omega[a.block_off[k]:a.block_off[k] + n * (n + 1) // 2] == 1.0)
    mom = np.nonzero(a.row_kind == 0)[0]
    dup = a.col[a.rowptr[mom] + 1]
    assert np.all(st.omega[dup] == 0.0) and np.all(st.inv_rep_s[dup] == 0.0)
    for c in range(st.rep.size):
        rows = st.row[st.ptr[c]:st.ptr[c + 1]]
        assert np.all(a.col[a.rowptr[rows]] == st.rep[c])
        assert abs(st.dsum[c] - st.inv_s2[st.ptr[c]:st.ptr[c + 1]].sum()) <= 1e-15 * st.dsum[c]
    # occurrences of each monomial over the full symmetric moment matrix
    # (diagonal once, off-diagonal twice) sum to s(nv, 4) monomials' worth:
    # sum over representatives of 1 / (omega s_r^2) = nM^2
    M0 = a.block_off[0]
    t = np.arange(nM * (nM + 1) // 2)
    j = np.floor((np.sqrt(8 * t + 1) - 1) / 2).astype(int)
    i = t - j * (j + 1) // 2
    s2 = np.where(i == j, 1.0, 0.5)
    reps = st.omega[M0 + t] > 0
    assert np.isclose(np.sum(1.0 / (st.omega[M0 + t][reps] * s2[reps])), nM * nM)


def test_rejects_malformed_input(S):
    p = wl.pendulum_problem(N=3, theta0=0.1)
    a = S.Problem(p).relax().export()

    def bad(match, **over):
        with pytest.raises(RuntimeError, match=match):
            _import(S, p, a, **over)

    # an A_mom row with a third entry
    r = int(np.nonzero(a.row_kind == 0)[0][0])
    rp = a.rowptr.copy()
    col = np.insert(a.col, rp[r + 1], a.col[rp[r + 1] - 1] + 1)
    val = np.insert(a.val, rp[r + 1], 0.5)
    rp[r + 1:] += 1
    bad("exactly two", rowptr=rp, col=col, val=val)
    # wrong svec scale on an A_mom row
    val = a.val.copy()
    val[a.rowptr[r]] *= 2.0
    bad("s_p X_p - s_r X_r", val=val)
    # a consensus row in the last clique
    rk = a.row_kind.copy()
    last = int(np.nonzero(a.row_clique == p.N - 1)[0][-1])
    rk[last] = 4
    bad("last clique", row_kind=rk)
    # a row of clique 0 reaching clique 2's moment block
    r0 = int(np.nonzero((a.row_clique == 0) & (a.row_kind == 2))[0][0])
    col = a.col.copy()
    col[a.rowptr[r0 + 1] - 1] = a.block_off[np.nonzero((a.block_clique == 2) & (a.block_kind == 0))[0][0]]
    bad("chain structure|strictly increasing", col=col)
    # columns out of order
    col = a.col.copy()
    e = a.rowptr[r0]
    col[e], col[e + 1] = col[e + 1], col[e]
    bad("strictly increasing", col=col)
    # a non-consensus row (phi_0) after a consensus row of the same clique
    rk = a.row_kind.copy()
    rk[int(np.nonzero((a.row_clique == 0) & (a.row_kind == 2))[0][-1])] = 4
    bad("close their clique", row_kind=rk)
    # blocks out of clique order, wrong moment size, NaN data
    bc = a.block_clique.copy()
    bc[0], bc[-1] = bc[-1], bc[0]
    bad("ordered by clique|moment block", block_clique=bc)
    bad("s\\(2 dx \\+ du, 2\\)", dx=p.dx + 1)
    Cn = a.C.copy()
    Cn[3] = np.nan
    bad("non-finite", C_=Cn)


def test_star_elimination_solves_A_At(S):
    """The y-solve's algebra on CPU, from the library's exported star data: the
    Gram A_o diag(omega) A_o^T of the other rows is the exact Schur complement of
    the A_mom rows in A A^T (Sherman-Morrison per star), and the star
    elimination -> Schur solve -> back substitution sequence (the steps of the
    GPU y-solve) returns (A_K A_K^T)^{-1} r_K of the row-reduced system (eq.
    solve-y1)."""
    import scipy.sparse as sp
    p = wl.pendulum_problem(N=3, theta0=0.1)
    sd = S.Problem(p).relax()
    a, st = sd.export(), sd.star_data()
    A = sp.csr_matrix((a.val, a.col, a.rowptr), shape=(len(a.rowptr) - 1, sd.nsvec))
    mom = a.row_kind == 0
    As, Ao = A[mom], A[~mom]
    Gss, Gso, Goo = (As @ As.T).toarray(), (As @ Ao.T).toarray(), (Ao @ Ao.T).toarray()
    schur = Goo - Gso.T @ np.linalg.solve(Gss, Gso)
    gram = (Ao @ sp.diags(st.omega) @ Ao.T).toarray()
    assert np.max(np.abs(schur - gram)) <= 1e-14 * np.max(np.abs(schur))
    # the whole solve on the kept rows, against the oracle's sparse LU
    red = OA.reduce(OR.relax(p))
    keep = red.keep
    assert np.all(keep[mom])                              # A_mom rows are always independent
    r = np.random.default_rng(5).standard_normal(A.shape[0])
    r[~keep] = 0.0
    rho = np.zeros(sd.nsvec)
    for c in range(st.rep.size):                          # star elimination (forward)
        q = st.row[st.ptr[c]:st.ptr[c + 1]]
        acc = np.sum(r[q] * st.inv_s2[st.ptr[c]:st.ptr[c + 1]])
        rho[st.rep[c]] = st.c[c] * acc / (1.0 + st.c[c] * st.dsum[c]) * st.inv_rep_s[st.rep[c]]
    oth = np.nonzero(~mom)[0]
    ko = keep[oth]
    t = r[oth] + Ao @ rho                                 # right-hand side of the Schur system
    y = np.zeros(A.shape[0])
    y[oth[ko]] = np.linalg.solve(gram[np.ix_(ko, ko)], t[ko])
    AoT = Ao.T.tocsr()
    for c in range(st.rep.size):                          # back substitution of the stars
        sl = slice(st.ptr[c], st.ptr[c + 1])
        q, is2 = st.row[sl], st.inv_s2[sl]
        rep = st.rep[c]
        gam = (AoT[rep] @ y[oth])[0] * st.inv_rep_s[rep]
        su = np.sum((r[q] + st.c[c] * gam) * is2)
        corr = st.c[c] * su / (1.0 + st.c[c] * st.dsum[c])
        y[q] = (r[q] + st.c[c] * gam) * is2 - is2 * corr
    want = OA.YSolver(red.A)(r[keep])
    assert np.linalg.norm(y[keep] - want) <= 1e-10 * np.linalg.norm(want)
    assert np.all(y[~keep] == 0.0)
