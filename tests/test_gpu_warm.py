"""Data-driven warm starts (Sec. 5, inverted pendulum with nearest-neighbour
warm starts): the device store, the combination against the oracle, and
warm-started solves through the solver and the serving batch."""
import numpy as np
import pytest

import workloads as wl
from oracle import warm as OW

from gpu_common import lib

pytestmark = pytest.mark.gpu

OPTS = dict(tol=1e-6, maxiter=20000, precision=2, check_every=10)
SCALE = np.array([0.1, 0.5])          # key = (theta0, omega0) / SCALE


def _relax(S, params, N=6):
    P = [S.Problem(wl.pendulum_problem(N=N, theta0=t, omega0=w)) for t, w in params]
    return P, [p.relax() for p in P]


def _database(S, params, N=6):
    P, sd = _relax(S, params, N)
    sv = S.Solver(sd, **OPTS)
    assert sv.solve() == S.STROM_OK
    store = S.WarmStore(2, sd[0].nsvec, len(params) + 4)
    for i, p in enumerate(params):
        assert store.add_from_solver(sv, i, np.array(p) / SCALE) == i
    return store, sv


def test_store_roundtrip_and_limits():
    S = lib()
    rng = np.random.default_rng(5)
    st = S.WarmStore(2, 50, 3)
    keys, X, Z = rng.normal(size=(3, 2)), rng.normal(size=(3, 50)), rng.normal(size=(3, 50))
    for j in range(3):
        assert st.add(keys[j], X[j], Z[j], 0.5 + j) == j
    assert len(st) == 3
    for j in range(3):
        k, x, z, sg = st.get(j)
        assert np.array_equal(k, keys[j]) and np.array_equal(x, X[j]) and np.array_equal(z, Z[j]) and sg == 0.5 + j
    with pytest.raises(RuntimeError, match="full"):
        st.add(keys[0], X[0], Z[0], 1.0)
    with pytest.raises(RuntimeError):
        S.WarmStore(2, 50, 1).add(keys[0], X[0], Z[0], -1.0)
    q = rng.normal(size=2)
    i1, w1 = st.query(q)
    i2, w2 = S.warm_select(keys, q)
    assert i1.tolist() == i2.tolist() and np.array_equal(w1, w2)


def test_solver_warm_start_is_the_oracle_combination():
    S = lib()
    P, sd = _relax(S, [(0.05, 0.1), (0.12, -0.2)])
    sv = S.Solver(sd, **OPTS)
    n = sd[0].nsvec
    rng = np.random.default_rng(6)
    keys = rng.uniform(-1, 1, size=(6, 2))
    Xs, Zs, sg = rng.normal(size=(6, n)), rng.normal(size=(6, n)), rng.uniform(0.1, 100, size=6)
    st = S.WarmStore(2, n, 6)
    for j in range(6):
        st.add(keys[j], Xs[j], Zs[j], sg[j])
    for q in ([0.1, 0.2], [5.0, -3.0], keys[3]):
        sv.warm_start(1, st, q)
        X, Z, y = sv.state(1)
        idx, w = OW.weights(keys, q)
        assert np.allclose(X, OW.combine(Xs, idx, w), rtol=0, atol=1e-14 * np.abs(Xs).max())
        assert np.allclose(Z, OW.combine(Zs, idx, w), rtol=0, atol=1e-14 * np.abs(Zs).max())
        assert not y.any()
        r = sv.result(1)
        assert r.iterations == 0 and abs(r.sigma - OW.sigma0(sg, idx, w)) <= 1e-14 * r.sigma
    # an empty store leaves the cold start
    sv.warm_start(0, S.WarmStore(2, n, 1), [0.1, 0.2])
    X, Z, _ = sv.state(0)
    assert not X.any() and not Z.any() and sv.result(0).sigma == 10.0


def test_warm_started_pendulum_starts_closer_and_reaches_the_same_optimum():
    S = lib()
    grid = [(t, w) for t in (0.04, 0.1, 0.16) for w in (-0.4, 0.0, 0.4)]
    store, _ = _database(S, grid)
    queries = [(0.07, 0.15), (0.13, -0.25), (0.09, 0.3)]
    P, sd = _relax(S, queries + queries)
    sv = S.Solver(sd, **OPTS)
    nq = len(queries)
    for i, q in enumerate(queries):
        sv.warm_start(nq + i, store, np.array(q) / SCALE)
    # after 20 iterations the warm-started instances are nearer the optimum
    sv.step(20)
    for i in range(nq):
        c, w = sv.result(i), sv.result(nq + i)
        assert max(w.eta_p, w.eta_d, w.eta_g) < max(c.eta_p, c.eta_d, c.eta_g)
    assert sv.solve() == S.STROM_OK
    certs = sv.certify_batch(P)
    for i in range(nq):
        cold, warm = sv.result(i), sv.result(nq + i)
        print("query %s: cold %d iterations, warm %d" % (queries[i], cold.iterations, warm.iterations))
        assert abs(warm.pobj - cold.pobj) <= 1e-5 * (1 + abs(cold.pobj))
        assert certs[nq + i].certified == certs[i].certified


def test_restart_from_own_solution_stops_at_once():
    # a key equal to a stored key takes that solution alone; Algorithm 1
    # started at its own fixed point meets tol in the first iteration
    S = lib()
    params = [(0.07, 0.15), (0.12, -0.2)]
    P, sd = _relax(S, params)
    opts = dict(OPTS, precision=0)
    sv = S.Solver(sd, **opts)
    assert sv.solve() == S.STROM_OK
    store = S.WarmStore(2, sd[0].nsvec, 2)
    for i, p in enumerate(params):
        store.add_from_solver(sv, i, np.array(p) / SCALE)
    again = S.Solver(sd, **opts)
    for i, p in enumerate(params):
        again.warm_start(i, store, np.array(p) / SCALE)
    assert again.solve() == S.STROM_OK
    for i in range(2):
        assert again.result(i).iterations <= 3
        assert abs(again.result(i).pobj - sv.result(i).pobj) <= 1e-6 * (1 + abs(sv.result(i).pobj))


def test_batch_keyed_request_equals_solver_warm_start():
    S = lib()
    grid = [(0.04, -0.4), (0.16, -0.4), (0.04, 0.4), (0.16, 0.4)]
    store, _ = _database(S, grid)
    q = (0.1, 0.1)
    P, sd = _relax(S, [q])
    batch = S.Batch(sd[0], 2, **OPTS)
    batch.set_warm(store, record=False)
    t = batch.submit_keyed(sd[0], np.array(q) / SCALE, P[0])
    for _ in range(100000):
        run, queued = batch.step(40)
        if run == 0 and queued == 0:
            break
    res, cert, _ = batch.poll(t)
    alone = S.Solver(sd, **OPTS)
    alone.warm_start(0, store, np.array(q) / SCALE)
    assert alone.solve() == S.STROM_OK
    a = alone.result(0)
    assert res.status == S.STROM_OK
    assert res.iterations == a.iterations and res.pobj == a.pobj and res.dobj == a.dobj and res.sigma == a.sigma
    assert len(store) == len(grid)          # not recording


def test_batch_records_converged_requests():
    S = lib()
    params = [(0.06, 0.1), (0.11, -0.1), (0.15, 0.2)]
    P, sd = _relax(S, params)
    store = S.WarmStore(2, sd[0].nsvec, 2)
    batch = S.Batch(sd[0], 1, **OPTS)
    with pytest.raises(RuntimeError, match="store"):
        batch.submit_keyed(sd[0], [0.0, 0.0])
    batch.set_warm(store, record=True)
    tickets = [batch.submit_keyed(s, np.array(p) / SCALE, pr) for s, p, pr in zip(sd, params, P)]
    for _ in range(100000):
        run, queued = batch.step(40)
        if run == 0 and queued == 0:
            break
    out = [batch.poll(t) for t in tickets]
    assert all(o is not None and o[0].status == S.STROM_OK for o in out)
    assert len(store) == 2                   # capacity 2: the third is not recorded
    for j in range(2):
        k, X, Z, sg = store.get(j)
        assert np.array_equal(k, np.array(params[j]) / SCALE) and sg == out[j][0].sigma
    # the second request started from the first one's solution (one slot, FIFO)
    alone = S.Solver([sd[1]], **OPTS)
    one = S.WarmStore(2, sd[0].nsvec, 1)
    k0, X0, Z0, s0 = store.get(0)
    one.add(k0, X0, Z0, s0)
    alone.warm_start(0, one, np.array(params[1]) / SCALE)
    alone.solve()
    assert alone.result(0).iterations == out[1][0].iterations and alone.result(0).pobj == out[1][0].pobj
