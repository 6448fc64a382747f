"""Continuous batching: every request's result is the same alone and in the mix."""
import pytest

import workloads as wl

from gpu_common import lib

pytestmark = pytest.mark.gpu


def test_served_equals_alone():
    S = lib()
    probs = wl.problem_batch("pendulum", 7, N=6)
    P = [S.Problem(p) for p in probs]
    sdps = [q.relax() for q in P]
    batch = S.Batch(sdps[0], 3, tol=1e-6, maxiter=20000, precision=S.STROM_PREC_MIXED, check_every=10)
    tickets = [batch.submit(sd, pr) for sd, pr in zip(sdps, P)]
    for _ in range(100000):
        run, queued = batch.step(40)
        if run == 0 and queued == 0:
            break
    out = [batch.poll(t) for t in tickets]
    assert all(o is not None for o in out)
    for i, (res, cert, lat) in enumerate(out):
        alone = S.Solver([sdps[i]], tol=1e-6, maxiter=20000, precision=S.STROM_PREC_MIXED, check_every=10)
        alone.solve()
        a = alone.result(0)
        assert res.status == S.STROM_OK and a.status == S.STROM_OK
        assert res.iterations == a.iterations
        assert res.pobj == a.pobj and res.dobj == a.dobj
        ca = alone.certify(0, P[i])
        assert cert is not None and cert.certified == ca.certified
        assert abs(cert.lower_bound - ca.lower_bound) <= 1e-12 * (1 + abs(ca.lower_bound))
        assert lat > 0


def test_submit_rejects_other_structure():
    S = lib()
    a = S.Problem(wl.pendulum_problem(N=4)).relax()
    b = S.Problem(wl.pendulum_problem(N=5)).relax()
    batch = S.Batch(a, 2)
    with pytest.raises(RuntimeError, match="structure"):
        batch.submit(b)
