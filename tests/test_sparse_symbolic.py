"""The symbolic analysis of the y-solve's sparse factor (host code, no GPU).

strom_sdp_factor_info reports the pattern of the Cholesky factor L of the
Gram S of the rows other than A_mom, in the canonical order of the row
reduction (cliques N..1, natural order inside a clique). Pinned here against
the elimination game played on the structural pattern of S, written out in
Python: eliminating vertex j joins all of its later neighbours, and the
column of L is that neighbour set. The per-group level schedules are checked
the same way.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as wl
from oracle import relax as OR

S = pytest.importorskip("paper_2406_05846_gb300")


def _lib_sdp(p):
    from paper_2406_05846_gb300 import build
    build.build()
    return S.Problem(p).relax()


def _structural(p):
    o = OR.relax(p)
    A = o.A.tocsr()
    other = np.nonzero(o.row_kind != OR.KIND_MOM)[0]
    # canonical order: cliques N..1, natural order inside
    order = np.concatenate([other[o.row_clique[other] == k] for k in range(o.N - 1, -1, -1)])
    Ao = abs(A[order])
    # weights: every column an other row touches is a representative or a localizing entry
    G = (Ao @ Ao.T).tocsr()
    groups = np.concatenate([[0], np.cumsum([np.sum(o.row_clique[other] == k) for k in range(o.N - 1, -1, -1)])])
    return G, groups


def _elimination_game(G):
    n = G.shape[0]
    adj = [set(G.indices[G.indptr[i]:G.indptr[i + 1]]) - {i} for i in range(n)]
    cols = []
    for j in range(n):
        later = {i for i in adj[j] if i > j}
        cols.append(sorted(later))
        for i in later:
            adj[i] |= later - {i}
    return cols


def _levels(cols, groups):
    n = len(cols)
    rows = [[] for _ in range(n)]
    for j, c in enumerate(cols):
        for i in c:
            rows[i].append(j)
    fwd = bwd = 0
    for g in range(len(groups) - 1):
        a, b = groups[g], groups[g + 1]
        lev = {}
        for i in range(a, b):
            lev[i] = max([lev[j] + 1 for j in rows[i] if j >= a], default=0)
        fwd += max(lev.values()) + 1
        lev = {}
        for j in range(b - 1, a - 1, -1):
            lev[j] = max([lev[i] + 1 for i in cols[j] if i < b], default=0)
        bwd += max(lev.values()) + 1
    return fwd, bwd


@pytest.mark.parametrize("make", [lambda: wl.toy_problem(N=3), lambda: wl.pendulum_problem(N=4, theta0=0.1),
                                  lambda: wl.cartpole_problem(N=2, x0=0.1, theta0=0.2)])
def test_factor_pattern_is_the_elimination_game(make):
    p = make()
    fi = _lib_sdp(p).factor_info()
    G, groups = _structural(p)
    cols = _elimination_game(G)
    assert fi["n_other"] == G.shape[0]
    assert fi["n_tail"] == groups[-2]
    assert fi["nnz_S"] == (G.nnz - G.shape[0]) // 2
    assert fi["nnz_L"] == sum(len(c) for c in cols)
    assert fi["max_col"] == max(len(c) for c in cols)
    assert fi["max_group"] == int(np.max(np.diff(groups)))
    fwd, bwd = _levels(cols, groups)
    assert (fi["levels_fwd"], fi["levels_bwd"]) == (fwd, bwd)
    # block bidiagonal by clique: a column's rows stay in its group or the next
    for g in range(len(groups) - 1):
        for j in range(groups[g], groups[g + 1]):
            assert all(i < groups[min(g + 2, len(groups) - 1)] for i in cols[j])
    dense = sum(int(m) * (int(m) + 1) // 2 for m in np.diff(groups))
    assert fi["dense_entries"] == dense
