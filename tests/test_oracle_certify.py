"""Pins of the oracle's certificate pieces (Theorem 1 iii, Sec. 2.2 extraction,
eq. valid-lowerbound with R_beta of App. C) — CPU only.

* Extraction from the rank-1 lifting of a feasible rollout returns that
  rollout exactly, with lambda_2 / lambda_1 = 0 in every clique.
* The rollout step (controls kept, states solved from each clique's
  equalities) reproduces an explicit simulation of the dynamics from states
  that were perturbed away from it.
* R_beta bounds trace(X_beta) of every lifted block over the variable box and
  is attained by the moment blocks at the corner z = (1, ..., 1) when R = 1.
* The lower bound is below the cost of every feasible trajectory, for any y.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import certify as CE
from oracle import relax as R
from oracle import sgs_admm as O

from test_oracle_relax import _pend_rollout
from test_oracle_robots import CP, cartpole_rollout


def _pendulum(N=4):
    p = wl.pendulum_problem(N=N, theta0=0.15)
    return p, _pend_rollout(p, np.random.default_rng(7).uniform(-1, 1, N))


def _cartpole(N=3):
    p = wl.cartpole_problem(N=N, x0=0.3, theta0=0.25, **CP)
    return p, cartpole_rollout(np.random.default_rng(8).uniform(-1, 1, N), 0.3, 0.25, **CP)


@pytest.mark.parametrize("make", [_pendulum, _cartpole])
def test_extraction_recovers_a_lifted_rollout(make):
    p, z = make()
    sdp = R.relax(p)
    ratios, zbar = CE.extract(p, sdp, R.lift_rank1(p, sdp, z))
    assert len(ratios) == p.N and np.max(np.abs(ratios)) < 1e-12
    assert np.max(np.abs(zbar - z)) < 1e-12


@pytest.mark.parametrize("make", [_pendulum, _cartpole])
def test_rollout_reconstructs_the_simulation(make):
    p, z = make()
    assert np.max(np.abs(CE.rollout(p, z) - z)) < 1e-13          # a feasible point is a fixed point
    noisy = z.copy()
    step = p.dx + p.du
    rng = np.random.default_rng(9)
    for k in range(1, p.N + 1):                                    # perturb every state after x_0
        noisy[k * step:k * step + p.dx] += 1e-3 * rng.standard_normal(p.dx)
    zhat = CE.rollout(p, noisy)
    assert np.max(np.abs(zhat - z)) < 1e-12
    hmax, gmin = CE.feasibility(p, zhat)
    assert hmax < 1e-12 and gmin >= 0


def test_r_beta_bounds_the_trace_and_is_attained():
    p, z = _pendulum(3)
    sdp = R.relax(p)
    rb = CE.r_beta(p, sdp)
    nv = p.nv
    for blk, r in zip(sdp.blocks, rb):
        if blk.kind == "M":
            assert r == R.s_count(nv, 2)
    # trace of every lifted block over random points of the box [-1, 1]^nz
    rng = np.random.default_rng(10)
    for _ in range(20):
        zz = rng.uniform(-1, 1, p.nz)
        X = R.lift_rank1(p, sdp, zz)
        for blk, r in zip(sdp.blocks, rb):
            M = R.smat(X[blk.offset:blk.offset + blk.n * (blk.n + 1) // 2], blk.n)
            assert np.trace(M) <= r * (1 + 1e-14)
    # the moment bound is attained at the corner of the box
    X = R.lift_rank1(p, sdp, np.ones(p.nz))
    for blk, r in zip(sdp.blocks, rb):
        if blk.kind == "M":
            M = R.smat(X[blk.offset:blk.offset + blk.n * (blk.n + 1) // 2], blk.n)
            assert abs(np.trace(M) - r) < 1e-12 * r


def test_lower_bound_is_below_every_feasible_cost():
    p = wl.pendulum_problem(N=3, theta0=0.15)
    red = O.reduce(R.relax(p))
    res = O.solve(red, O.Options(tol=1e-8, maxiter=20000))
    rng = np.random.default_rng(11)
    costs = [p.objective(_pend_rollout(p, rng.uniform(-1, 1, 3))) for _ in range(50)]
    for t in (0.0, 0.5, 1.0, 1.5):
        # the bound holds for every multiplier y, not only at the optimum
        c = CE.certify(p, red, res.X, t * res.y)
        assert c.lower_bound <= min(costs) + 1e-12
    c = CE.certify(p, red, res.X, res.y)
    assert c.lower_bound <= res.pobj + 1e-6 * (1 + abs(res.pobj))
    assert c.feasible and c.phat >= c.lower_bound and c.xi >= 0
