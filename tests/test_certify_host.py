"""The library's host certificate (strom_certify_host) against the oracle's
certify(): extraction, rollout, R_beta lower bound and verdict from the same
eigen data, on CPU (Theorem 1 iii, Sec. 2.2, eq. valid-lowerbound, eq.
suboptimality-gap). The eigen data come from numpy on the oracle's solution;
on the GPU path they come from the library's Jacobi kernels instead."""
import numpy as np
import pytest

import workloads as wl
from oracle import certify as CE
from oracle import relax as R
from oracle import sgs_admm as O


@pytest.fixture(scope="module")
def S():
    from paper_2406_05846_gb300 import build
    build.build()
    import paper_2406_05846_gb300 as S
    S.lib()
    return S


def _eig_data(red, X, y):
    """Per block of X: ascending eigenvalues and the top eigenvector; per block
    of Z = C - A^T y: ascending eigenvalues; all packed block after block."""
    sdp = red.sdp
    Z = sdp.C - red.A.T @ y
    lamX, topX, lamZ = [], [], []
    for b in sdp.blocks:
        t = b.n * (b.n + 1) // 2
        w, V = np.linalg.eigh(R.smat(X[b.offset:b.offset + t], b.n))
        lamX.append(w)
        topX.append(V[:, -1])
        lamZ.append(np.linalg.eigvalsh(R.smat(Z[b.offset:b.offset + t], b.n)))
    bn = [b.n for b in sdp.blocks]
    bk = [0 if b.kind == "M" else 1 for b in sdp.blocks]
    bc = [b.clique for b in sdp.blocks]
    return bn, bk, bc, np.concatenate(lamX), np.concatenate(topX), np.concatenate(lamZ), float(red.b @ y)


@pytest.mark.parametrize("which", ["toy", "pendulum"])
def test_host_certificate_matches_oracle(S, which):
    # the toy problem has R = 2, so R_beta's power of max(1, R) is exercised
    p = wl.toy_problem(N=3) if which == "toy" else wl.pendulum_problem(N=3, theta0=0.15)
    red = O.reduce(R.relax(p))
    res = O.solve(red, O.Options(tol=1e-9, maxiter=40000))
    want = CE.certify(p, red, res.X, res.y)
    got = S.certify_host(S.Problem(p), *_eig_data(red, res.X, res.y))
    assert abs(got.max_ratio - want.max_ratio) <= 1e-12
    assert abs(got.lower_bound - want.lower_bound) <= 1e-10 * (1 + abs(want.lower_bound))
    assert abs(got.phat - want.phat) <= 1e-10 * (1 + abs(want.phat))
    assert abs(got.xi - want.xi) <= 1e-10
    assert np.max(np.abs(got.zbar - want.zbar)) <= 1e-9
    assert np.max(np.abs(got.zhat - want.zhat)) <= 1e-9
    assert (got.feasible, got.rank_one, got.certified) == (want.feasible, want.rank_one, want.certified)


def test_host_certificate_of_a_lifted_rollout(S):
    """A rank-1 lifting of a feasible rollout with y = 0: ratios 0, the rollout
    comes back exactly, and the bound is sum_beta R_beta min(0, lambda_min(C_beta))."""
    from test_oracle_relax import _pend_rollout
    p = wl.pendulum_problem(N=4, theta0=0.1)
    z = _pend_rollout(p, np.random.default_rng(3).uniform(-1, 1, 4))
    sdp = R.relax(p)
    red = O.reduce(sdp)
    X = R.lift_rank1(p, sdp, z)
    y = np.zeros(red.m)
    got = S.certify_host(S.Problem(p), *_eig_data(red, X, y))
    assert got.max_ratio < 1e-12 and got.rank_one and got.feasible
    assert np.max(np.abs(got.zbar - z)) < 1e-12 and np.max(np.abs(got.zhat - z)) < 1e-12
    assert abs(got.phat - p.objective(z)) < 1e-12
    rb = CE.r_beta(p, sdp)
    lmin = [np.linalg.eigvalsh(R.smat(sdp.C[b.offset:b.offset + b.n * (b.n + 1) // 2], b.n))[0] for b in sdp.blocks]
    assert abs(got.lower_bound - float(np.sum(rb * np.minimum(0.0, lmin)))) <= 1e-12 * (1 + abs(got.lower_bound))


def test_host_certificate_rejects_mismatched_blocks(S):
    from paper_2406_05846_gb300._native import StromError
    p = wl.pendulum_problem(N=2, theta0=0.1)
    red = O.reduce(R.relax(p))
    bn, bk, bc, lx, tx, lz, by = _eig_data(red, np.zeros(red.sdp.nsvec), np.zeros(red.m))
    P = S.Problem(p)
    with pytest.raises(StromError):                      # a localizing block missing
        S.certify_host(P, bn[:-1], bk[:-1], bc[:-1], lx[:-bn[-1]], tx[:-bn[-1]], lz[:-bn[-1]], by)
    bad = list(bc)
    bad[0] = 5                                           # clique out of range
    with pytest.raises(StromError):
        S.certify_host(P, bn, bk, bad, lx, tx, lz, by)
    with pytest.raises(ValueError):                      # eigen data of the wrong length
        S.certify_host(P, bn, bk, bc, lx[:-1], tx, lz, by)
