"""The sparse factor of the y-solve (eq. cholesky on the star-eliminated
system) against the FP64 oracle: row reduction, y-solve, iterations.

The sparse factor takes the same pivot decisions as the oracle's row
reduction (cliques N..1, natural order inside a clique), so keep masks must be
identical and y must agree to the y-solve's FP64 bar. Where the oracle's row
reduction is too slow (the rigid body's first clique has 11,856 other rows),
properties that hold at any size are checked instead: the backward error of
the solve, the kept rows are independent and every dropped row lies in their
span.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as wl
from oracle import relax as OR
from oracle import sgs_admm as OA

from gpu_common import assert_close, dev, host, lib, torch

pytestmark = pytest.mark.gpu

YTOL = 1e-10   # relative, the y-solve's FP64 bar


def _solve(solver, r):
    rd = dev(r)
    yd = torch.zeros_like(rd)
    solver.kernel_solve(rd.data_ptr(), yd.data_ptr())
    return host(yd)


def _reference_y(red, r):
    """The oracle's y = (A_K A_K^T)^{-1} r_K with two steps of iterative
    refinement on the exact sparse product (the unrefined sparse-LU solution
    carries the conditioning of A_K A_K^T, about 1e-10 relative on the
    cart-pole at N = 50)."""
    ys = OA.YSolver(red.A)
    y = ys(r)
    for _ in range(2):
        y = y + ys(r - red.A @ (red.A.T @ y))
    return y


def _check_y(got, want, keep, tol=YTOL):
    assert np.all(got[~keep] == 0.0)
    g = got[keep]
    assert np.linalg.norm(g - want) <= tol * np.linalg.norm(want), np.linalg.norm(g - want) / np.linalg.norm(want)
    assert np.max(np.abs(g - want)) <= tol * np.max(np.abs(want))


def test_sparse_pendulum_matches_oracle():
    S = lib()
    probs = [wl.pendulum_problem(N=10, theta0=t) for t in (0.1, -0.17, 0.02)]
    solver = S.Solver([S.Problem(p).relax() for p in probs], factor=S.STROM_FACTOR_SPARSE)
    r = np.random.default_rng(2).standard_normal(solver.m_total)
    y = _solve(solver, r)
    for i, p in enumerate(probs):
        red = OA.reduce(OR.relax(p))
        assert np.array_equal(solver.kept_rows(i), red.keep)
        so, ro = solver.offsets(i)
        _check_y(y[ro:ro + red.sdp.m], OA.YSolver(red.A)(r[ro:ro + red.sdp.m][red.keep]), red.keep)


def test_sparse_equals_dense():
    S = lib()
    probs = [wl.pendulum_problem(N=8, theta0=t) for t in (0.05, -0.12)]
    sd = [S.Problem(p).relax() for p in probs]
    a = S.Solver(sd, factor=S.STROM_FACTOR_DENSE)
    b = S.Solver(sd, factor=S.STROM_FACTOR_SPARSE)
    for i in range(len(sd)):
        assert np.array_equal(a.kept_rows(i), b.kept_rows(i))
    r = np.random.default_rng(3).standard_normal(a.m_total)
    ya, yb = _solve(a, r), _solve(b, r)
    # two summation orders on a matrix of condition number ~1e7: the y-solve bar
    assert_close(yb, ya, YTOL, what="sparse vs dense y")


def test_sparse_cartpole_matches_oracle():
    S = lib()
    p = wl.cartpole_problem(N=3, x0=0.2, theta0=0.1)
    red = OA.reduce(OR.relax(p))
    solver = S.Solver([S.Problem(p).relax()], tol=1e-12, maxiter=25, check_every=1, precision=S.STROM_PREC_FP64,
                      factor=S.STROM_FACTOR_SPARSE)
    assert np.array_equal(solver.kept_rows(0), red.keep)
    r = np.random.default_rng(4).standard_normal(solver.m_total)
    _check_y(_solve(solver, r), OA.YSolver(red.A)(r[red.keep]), red.keep)
    solver.step(25)
    X, Sg, _ = solver.state(0)
    ref = OA.solve(red, OA.Options(tol=1e-12, maxiter=25))
    assert_close(X, ref.X, 1e-9, what="X")
    assert_close(Sg, ref.S, 1e-9, floor=1.0, what="S")


def test_sparse_cartpole_full_horizon_shared_tail():
    """Cart-pole at the configuration's N = 50: three instances share the
    factor of cliques 2..N (one owner, two that factorise their first clique
    only); keep masks and y against the oracle for the owner and one other."""
    S = lib()
    probs = wl.problem_batch("cartpole", 3, N=50)
    solver = S.Solver([S.Problem(p).relax() for p in probs], factor=S.STROM_FACTOR_SPARSE)
    r = np.random.default_rng(5).standard_normal(solver.m_total)
    y = _solve(solver, r)
    for i in (0, 2):
        red = OA.reduce(OR.relax(probs[i]))
        assert np.array_equal(solver.kept_rows(i), red.keep)
        so, ro = solver.offsets(i)
        rk = r[ro:ro + red.sdp.m][red.keep]
        ref = _reference_y(red, rk)
        got = y[ro:ro + red.sdp.m]
        # the conditioning of A_K A_K^T here puts every FP64 normal-equation
        # solve near 1e-10: the bar is 1e-10 or the oracle's own sparse-LU
        # error against the refined reference, whichever is larger, with a
        # backward error of at most 1e-12
        plain = OA.YSolver(red.A)(rk)
        e_lu = max(np.linalg.norm(plain - ref) / np.linalg.norm(ref),
                   np.max(np.abs(plain - ref)) / np.max(np.abs(ref)))
        back = np.linalg.norm(red.A @ (red.A.T @ got[red.keep]) - rk) / np.linalg.norm(rk)
        assert back <= 1e-12, back
        _check_y(got, ref, red.keep, tol=max(YTOL, e_lu))


@pytest.mark.parametrize("tile", ["2", "4", "8"])
def test_sparse_tiles_bit_identical(tile, monkeypatch):
    """Tiles of instances sharing the tail give bit-identical y to one
    instance per CTA (9 instances: a ragged last tile)."""
    S = lib()
    probs = [wl.pendulum_problem(N=6, theta0=t) for t in np.linspace(-0.19, 0.18, 9)]
    sd = [S.Problem(p).relax() for p in probs]
    monkeypatch.setenv("STROM_TILE_R", "1")
    one = S.Solver(sd, factor=S.STROM_FACTOR_SPARSE)
    monkeypatch.setenv("STROM_TILE_R", tile)
    multi = S.Solver(sd, factor=S.STROM_FACTOR_SPARSE)
    r = np.random.default_rng(7).standard_normal(one.m_total)
    assert np.array_equal(_solve(one, r), _solve(multi, r))


def test_sparse_batch_equals_alone():
    S = lib()
    probs = [wl.cartpole_problem(N=3, x0=x, theta0=t) for x, t in ((0.1, 0.2), (-0.3, -0.1), (0.4, 0.05))]
    sd = [S.Problem(p).relax() for p in probs]
    batch = S.Solver(sd, tol=1e-12, maxiter=60, check_every=60, precision=S.STROM_PREC_FP64,
                     factor=S.STROM_FACTOR_SPARSE)
    batch.step(60)
    for i, p in enumerate(probs):
        alone = S.Solver([S.Problem(p).relax()], tol=1e-12, maxiter=60, check_every=60,
                         precision=S.STROM_PREC_FP64, factor=S.STROM_FACTOR_SPARSE)
        alone.step(60)
        xa, _, ya = alone.state(0)
        xb, _, yb = batch.state(i)
        assert np.array_equal(xa, xb) and np.array_equal(ya, yb)


def test_sparse_rigid_body_solve_properties():
    """Rigid body (16-variable cliques, 153 x 153 moment blocks), horizon 2,
    three disks: the y-solve's backward error, and the kept rows form a basis
    of the row space (independent, spanning every dropped row)."""
    S = lib()
    p = wl.rigid_body_problem(N=2, disks=[(0.5, 0.5, 0.4), (1.0, -1.0, 0.5), (-0.5, 1.0, 0.3)])
    solver = S.Solver([S.Problem(p).relax()], factor=S.STROM_FACTOR_SPARSE)
    o = OR.relax(p)
    keep = solver.kept_rows(0).astype(bool)
    A = o.A.tocsr()
    AK = A[keep]
    G = (AK @ AK.T).tocsc()
    lu = spla.splu(G, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0, options=dict(SymmetricMode=True))
    assert np.all(lu.U.diagonal() > 0)                     # A_K A_K^T is positive definite
    dropped = np.nonzero(~keep)[0]
    assert len(dropped) > 0
    sample = np.random.default_rng(9).choice(dropped, size=min(400, len(dropped)), replace=False)
    drop = A[sample]
    coef = lu.solve((AK @ drop.T).toarray())
    resid = (AK.T @ coef - drop.T.toarray())
    assert np.max(np.linalg.norm(resid, axis=0) / np.linalg.norm(drop.toarray(), axis=1)) <= 1e-8
    r = np.random.default_rng(8).standard_normal(solver.m_total)
    y = _solve(solver, r)
    assert np.all(y[~keep] == 0.0)
    # normwise backward error ||G y - r|| / (||G|| ||y|| + ||r||) of the solve:
    # the kept pivots reach down to rank_tol (1e-8) of their row norms, so
    # ||y|| may be far above ||r||
    yk, rk = y[keep], r[keep]
    eta = np.linalg.norm(G @ yk - rk) / (spla.norm(G) * np.linalg.norm(yk) + np.linalg.norm(rk))
    assert eta <= 1e-13, eta
