"""Failure paths of the solver, driven from the host without faulting the GPU:
a non-finite warm state in one instance, a spent time budget, and a serving
budget larger than the device. Also the y-solve autotuner, run for real."""
import numpy as np
import pytest

import workloads as wl

from gpu_common import lib

pytestmark = pytest.mark.gpu


def _pendulums(S, n, N=6):
    probs = wl.problem_batch("pendulum", n, N=N)
    return [S.Problem(p).relax() for p in probs]


def test_nan_in_one_instance_is_isolated():
    """A warm state with a NaN entry given to instance 1 of 3: that instance
    ends with STROM_ERR_NUMERICAL, strom_solve reports it, and instances 0
    and 2 are bit-identical to a run without it."""
    S = lib()
    sd = _pendulums(S, 3)
    opts = dict(tol=1e-6, maxiter=4000, precision=S.STROM_PREC_MIXED, check_every=50)
    clean = S.Solver(sd, **opts)
    assert clean.solve() == S.STROM_OK
    bad = S.Solver(sd, **opts)
    X0 = np.zeros(sd[1].nsvec)
    X0[17] = np.nan
    bad.reset(1, X0=X0, S0=np.zeros(sd[1].nsvec))
    with pytest.raises(S.StromError) as e:
        bad.solve()
    assert e.value.status == S.STROM_ERR_NUMERICAL
    assert bad.result(1).status == S.STROM_ERR_NUMERICAL
    for i in (0, 2):
        a, b = clean.result(i), bad.result(i)
        assert b.status == S.STROM_OK
        assert a.iterations == b.iterations and a.pobj == b.pobj and a.dobj == b.dobj
        xa, sa, ya = clean.state(i)
        xb, sb, yb = bad.state(i)
        assert np.array_equal(xa, xb) and np.array_equal(sa, sb) and np.array_equal(ya, yb)


def test_time_budget_returns_timeout_with_valid_state():
    """A budget far below one check interval: strom_solve stops after the
    first check_every iterations with STROM_ERR_TIMEOUT, and the state and
    results of those iterations are finite and readable; a second call
    continues from them."""
    S = lib()
    sd = _pendulums(S, 2, N=10)
    sv = S.Solver(sd, tol=1e-6, maxiter=20000, precision=S.STROM_PREC_FP64, check_every=25, time_budget_s=1e-6)
    with pytest.raises(S.StromError) as e:
        sv.solve()
    assert e.value.status == S.STROM_ERR_TIMEOUT
    for i in range(2):
        r = sv.result(i)
        assert r.iterations == 25 and r.status == S.STROM_MAXITER
        assert np.isfinite([r.pobj, r.dobj, r.eta_p, r.eta_d, r.eta_g]).all()
        X, Sg, y = sv.state(i)
        assert np.isfinite(X).all() and np.isfinite(Sg).all() and np.isfinite(y).all()
    with pytest.raises(S.StromError) as e:
        sv.solve()
    assert e.value.status == S.STROM_ERR_TIMEOUT
    assert sv.result(0).iterations == 50


def test_batch_budget_beyond_the_device_is_oom():
    """A serving batch asked to fit in more bytes than the device has is
    refused with STROM_ERR_OOM before anything is allocated; a budget below
    one slot is INVALID; a budget of a few slots gives that many slots."""
    S = lib()
    import torch
    tmpl = _pendulums(S, 1)[0]
    per = S.Batch.slot_bytes(tmpl, precision=S.STROM_PREC_MIXED)
    assert per > 0
    total = torch.cuda.mem_get_info()[1]
    with pytest.raises(S.StromError) as e:
        S.Batch.with_budget(tmpl, 4 * total, precision=S.STROM_PREC_MIXED)
    assert e.value.status == S.STROM_ERR_OOM
    with pytest.raises(S.StromError) as e:
        S.Batch.with_budget(tmpl, per // 2, precision=S.STROM_PREC_MIXED)
    assert e.value.status == S.STROM_ERR_INVALID
    f = S.Batch.footprint(tmpl, precision=S.STROM_PREC_MIXED)
    assert f["slot"] == per
    b = S.Batch.with_budget(tmpl, f["base"] + f["transient"] + int(3.5 * per), precision=S.STROM_PREC_MIXED)
    assert b.slots == 3


def test_autotuner_times_every_tile_and_keeps_results():
    """strom_solver_tune on 40 pendulum instances sharing the tail factor:
    every y-solve launch shape is timed and the fastest kept; every
    eigensolver size class in use gets a thread count with a time; the
    iterations after tuning agree with an untuned solver's to rounding (the
    y-solve shapes give bit-identical arithmetic, the eigensolver's thread
    count only reorders the sum of its stopping test)."""
    S = lib()
    from gpu_common import assert_close
    sd = _pendulums(S, 40)
    opts = dict(tol=1e-12, maxiter=60, precision=S.STROM_PREC_MIXED, check_every=60)
    a = S.Solver(sd, **opts)
    times, tile = a.tune(reps=3)
    assert set(times) >= {1, 2} and all(t > 0 for t in times.values())
    assert times[tile] == min(times.values())
    # pendulum blocks: 36 x 36 moment (class n <= 40), 8 x 8 localizing (n <= 16)
    for prec in ("fp64", "fp32"):
        got = a.eig_tuning[prec]
        assert set(got) == {0, 1}, got
        assert all(th in (32, 64, 128, 256) and ms > 0 for th, ms in got.values())
    b = S.Solver(sd, **opts)
    a.step(60)
    b.step(60)
    for i in (0, 17, 39):
        xa, _, ya = a.state(i)
        xb, _, yb = b.state(i)
        assert_close(xa, xb, 1e-5, what=("X", i))
