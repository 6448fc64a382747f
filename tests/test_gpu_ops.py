"""A(X), A^T(y), row reduction and the y-solve vs the oracle (FP64)."""
import numpy as np
import pytest

import workloads as wl
from oracle import relax as OR
from oracle import sgs_admm as OA

from gpu_common import assert_close, dev, host, lib, torch

pytestmark = pytest.mark.gpu


def _batch(S, problems, **opt):
    sdps = [S.Problem(p).relax() for p in problems]
    return S.Solver(sdps, **opt), [OR.relax(p) for p in problems]


@pytest.fixture(scope="module")
def pend_batch():
    S = lib()
    probs = [wl.pendulum_problem(N=10, theta0=t) for t in (0.1, -0.17, 0.02)]
    solver, osdps = _batch(S, probs)
    return S, probs, solver, osdps


def test_A_and_At(pend_batch):
    S, probs, solver, osdps = pend_batch
    rng = np.random.default_rng(1)
    x = rng.standard_normal(solver.nsvec_total)
    y = rng.standard_normal(solver.m_total)
    xd, yd = dev(x), dev(y)
    ax = torch.zeros(solver.m_total, dtype=torch.float64, device="cuda:0")
    aty = torch.zeros(solver.nsvec_total, dtype=torch.float64, device="cuda:0")
    solver.kernel_A(xd.data_ptr(), ax.data_ptr())
    solver.kernel_At(yd.data_ptr(), aty.data_ptr())
    ax, aty = host(ax), host(aty)
    for i, o in enumerate(osdps):
        so, ro = solver.offsets(i)
        want = o.A @ x[so:so + o.nsvec]
        assert np.max(np.abs(ax[ro:ro + o.m] - want)) <= 1e-13 * np.max(np.abs(want))
        want_t = o.A.T @ y[ro:ro + o.m]
        assert np.max(np.abs(aty[so:so + o.nsvec] - want_t)) <= 1e-13 * np.max(np.abs(want_t))


@pytest.mark.parametrize("which", ["pendulum", "toy", "cartpole"])
def test_row_reduction_matches_oracle(which):
    S = lib()
    if which == "pendulum":
        probs = [wl.pendulum_problem(N=10, theta0=0.1), wl.pendulum_problem(N=4, theta0=-0.05)]
    elif which == "toy":
        probs = [wl.toy_problem(N=3), wl.toy_problem(N=5)]
    else:
        probs = [wl.cartpole_problem(N=2, x0=0.1, theta0=0.2)]
    solver, osdps = _batch(S, probs)
    for i, o in enumerate(osdps):
        keep, _ = OA.reduce_rows(o)
        assert np.array_equal(solver.kept_rows(i), keep)


def test_ysolve_matches_oracle(pend_batch):
    S, probs, solver, osdps = pend_batch
    rng = np.random.default_rng(2)
    r = rng.standard_normal(solver.m_total)
    rd = dev(r)
    yd = torch.zeros_like(rd)
    solver.kernel_solve(rd.data_ptr(), yd.data_ptr())
    y = host(yd)
    for i, o in enumerate(osdps):
        red = OA.reduce(o)
        so, ro = solver.offsets(i)
        want = OA.YSolver(red.A)(r[ro:ro + o.m][red.keep])
        got = y[ro:ro + o.m]
        assert np.all(got[~red.keep] == 0.0)
        assert_close(got[red.keep], want, 1e-10, what=("y", i))


_CART = {}


def _cartpole_case():
    """Cart-pole, horizon 2 (11-variable cliques: 78x78 moment and 12x12
    localizing blocks), with its oracle row reduction computed once."""
    if not _CART:
        p = wl.cartpole_problem(N=2, x0=0.2, theta0=0.1)
        o = OR.relax(p)
        _CART["p"], _CART["red"] = p, OA.reduce(o)
    return _CART["p"], _CART["red"]


def test_cartpole_ysolve_and_iterations_match_oracle():
    S = lib()
    p, red = _cartpole_case()
    solver = S.Solver([S.Problem(p).relax()], tol=1e-12, maxiter=25, check_every=1, precision=S.STROM_PREC_FP64)
    assert np.array_equal(solver.kept_rows(0), red.keep)
    # y-solve on a random right-hand side
    rng = np.random.default_rng(4)
    r = rng.standard_normal(solver.m_total)
    rd = dev(r)
    yd = torch.zeros_like(rd)
    solver.kernel_solve(rd.data_ptr(), yd.data_ptr())
    y = host(yd)
    want = OA.YSolver(red.A)(r[red.keep])
    assert_close(y[red.keep], want, 1e-10, what="y")
    # the first 25 iterations of Algorithm 1
    solver.step(25)
    X, Sg, _ = solver.state(0)
    ref = OA.solve(red, OA.Options(tol=1e-12, maxiter=25))
    assert_close(X, ref.X, 1e-9, what="X")
    assert_close(Sg, ref.S, 1e-9, floor=1.0, what="S")


@pytest.mark.parametrize("tile", ["2", "4", "8"])
def test_multi_rhs_solve_matches_single(tile, monkeypatch):
    """The tiled multi-right-hand-side chain solve (shared factor of cliques
    2..N) gives bit-identical y to the one-instance-per-CTA solve, and both
    match the oracle; 9 instances leave a ragged last tile."""
    S = lib()
    probs = [wl.pendulum_problem(N=6, theta0=t) for t in np.linspace(-0.19, 0.18, 9)]
    sd = [S.Problem(p).relax() for p in probs]
    rng = np.random.default_rng(7)
    monkeypatch.setenv("STROM_TILE_R", "1")
    one = S.Solver(sd, precision=S.STROM_PREC_FP64)
    monkeypatch.setenv("STROM_TILE_R", tile)
    multi = S.Solver(sd, precision=S.STROM_PREC_FP64)
    r = rng.standard_normal(one.m_total)
    rd = dev(r)
    y1, y2 = torch.zeros_like(rd), torch.zeros_like(rd)
    one.kernel_solve(rd.data_ptr(), y1.data_ptr())
    multi.kernel_solve(rd.data_ptr(), y2.data_ptr())
    a, b = host(y1), host(y2)
    assert np.array_equal(a, b)
    for i in (0, 8):
        red = OA.reduce(OR.relax(probs[i]))
        so, ro = one.offsets(i)
        want = OA.YSolver(red.A)(r[ro:ro + red.sdp.m][red.keep])
        assert_close(b[ro:ro + red.sdp.m][red.keep], want, 1e-10, what=("y", i))


def test_raw_csr_products_match_oracle():
    """strom_kernel_spmv_csr on the oracle's A and A^T given as raw device
    arrays (int64 row pointers, int32 columns, FP64 values): A(X) and A^*(y)
    against SciPy's products of the same matrices, entry by entry."""
    S = lib()
    o = OR.relax(wl.pendulum_problem(N=6, theta0=0.08))
    rng = np.random.default_rng(11)
    for M in (o.A.tocsr(), o.A.T.tocsr()):
        M.sort_indices()
        x = rng.standard_normal(M.shape[1])
        rp = torch.tensor(M.indptr.astype(np.int64), device="cuda:0")
        ci = torch.tensor(M.indices.astype(np.int32), device="cuda:0")
        va = torch.tensor(M.data.astype(np.float64), device="cuda:0")
        xd = dev(x)
        yd = torch.zeros(M.shape[0], dtype=torch.float64, device="cuda:0")
        S.kernel_spmv_csr(rp.data_ptr(), ci.data_ptr(), va.data_ptr(), M.shape[0], xd.data_ptr(), yd.data_ptr())
        assert_close(host(yd), M @ x, 1e-13, what=M.shape)
