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


def _alone(S, sd, opts):
    sv = S.Solver([sd], **opts)
    sv.solve()
    return sv.result(0)


def _drain(srv, tickets):
    out = {}
    for _ in range(100000):
        run, waiting = srv.step(40)
        for t in tickets:
            if t not in out:
                o = srv.poll(t)
                if o is not None:
                    out[t] = o
        if run == 0 and waiting == 0:
            break
    return out


def test_server_mixed_structures_equal_alone():
    """Pendulums of horizons 6 and 8 and cart-poles of horizon 3 behind one
    server: three classes, one batch each, stepped at the same time; every
    result is the one the request gets when solved alone."""
    S = lib()
    opts = dict(tol=1e-6, maxiter=20000, precision=S.STROM_PREC_MIXED, check_every=10)
    probs = (wl.problem_batch("pendulum", 4, N=6) + wl.problem_batch("pendulum", 3, N=8)
             + wl.problem_batch("cartpole", 2, N=3))
    P = [S.Problem(p) for p in probs]
    sdps = [q.relax() for q in P]
    srv = S.Server(2 << 30, 3, **opts)
    tickets = [srv.submit(sd, pr) for sd, pr in zip(sdps, P)]
    out = _drain(srv, tickets)
    assert len(out) == len(tickets)
    classes, used = srv.info()
    assert len(classes) == 3 and all(c["shared_tail"] == 1 for c in classes)
    assert sorted(c["N"] for c in classes) == [3, 6, 8]
    assert 0 < used <= 2 << 30
    for t, sd, pr in zip(tickets, sdps, P):
        res, cert, lat = out[t]
        a = _alone(S, sd, opts)
        assert res.status == S.STROM_OK and a.status == S.STROM_OK
        assert res.iterations == a.iterations and res.pobj == a.pobj and res.dobj == a.dobj
        assert cert is not None and lat > 0


def test_server_budget_evicts_idle_batches():
    """A budget that holds one class's batch at a time: the second structure
    waits, its batch is made once the first class is idle (the first batch
    is destroyed to make room), and every result is still the one of solving
    alone; a budget above the device's free memory is refused (OOM)."""
    S = lib()
    import torch
    opts = dict(tol=1e-6, maxiter=20000, precision=S.STROM_PREC_MIXED, check_every=10)
    pa = wl.problem_batch("pendulum", 2, N=6)
    pb = wl.problem_batch("pendulum", 2, N=9)
    P = [S.Problem(p) for p in pa + pb]
    sdps = [q.relax() for q in P]
    fa = S.Batch.footprint(sdps[0], **opts)
    fb = S.Batch.footprint(sdps[2], **opts)
    need = [f["base"] + f["transient"] + 2 * f["slot"] for f in (fa, fb)]
    budget = max(need) + min(fa["slot"], fb["slot"]) // 2
    assert budget < sum(need)
    srv = S.Server(budget, 2, **opts)
    tickets = [srv.submit(sd, pr) for sd, pr in zip(sdps, P)]
    run, waiting = srv.step(40)
    assert waiting == 2      # the second structure found no room
    out = _drain(srv, tickets)
    assert len(out) == 4
    classes, _ = srv.info()
    assert [c["batches_created"] for c in classes] == [1, 1]
    assert classes[0]["slots"] == 0          # evicted
    for t, sd in zip(tickets, sdps):
        res, _, _ = out[t]
        a = _alone(S, sd, opts)
        assert res.iterations == a.iterations and res.pobj == a.pobj
    total = torch.cuda.mem_get_info()[1]
    with pytest.raises(S.StromError) as e:
        S.Server(4 * total, 2, **opts)
    assert e.value.status == S.STROM_ERR_OOM
