"""Whole-solve parity on seeded batches: every instance of a batched solve,
and a sample of served requests, against the FP64 oracle's reference solves.

The references are in tests/golden/oracle_refs.json, written by
tests/golden/make_oracle_refs.py, which calls only oracle/: Algorithm 1 run to
max(eta_p, eta_d, eta_g) <= 1e-8, then the oracle's certificate. A GPU solve
stopped at 1e-6 must have its objective within 1e-6 (relative) of that
reference, and the same rank-1 verdict, feasibility of the rollout and
certificate, except for instances whose lambda_2 / lambda_1 lies in the
borderline band [5e-5, 2e-4] around the 1e-4 threshold, where two correct
solves may fall on either side.
"""
import json
import os

import numpy as np
import pytest

import workloads as wl

from gpu_common import lib

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
REFS = os.path.join(HERE, "golden", "oracle_refs.json")
BAND = (5e-5, 2e-4)
OBJ_TOL = 1e-6


def _refs(kind, idx):
    if not os.path.exists(REFS):
        pytest.skip("no oracle references (tests/golden/make_oracle_refs.py)")
    refs = json.load(open(REFS)).get(kind, {})
    missing = [i for i in idx if str(i) not in refs]
    if missing:
        pytest.skip("oracle references missing for %s %s" % (kind, missing))
    return [refs[str(i)] for i in idx]


def _check(S, res, cert, ref, what):
    assert ref["converged"], (what, ref)
    assert res.status == S.STROM_OK, (what, res)
    assert max(res.eta_p, res.eta_d, res.eta_g) <= 1e-6, (what, res)
    rel = abs(res.pobj - ref["pobj"]) / (1.0 + abs(ref["pobj"]))
    assert rel <= OBJ_TOL, (what, res.pobj, ref["pobj"], rel)
    assert res.m_kept == ref["m_kept"], what
    if cert is None:
        return
    border = BAND[0] <= ref["max_ratio"] <= BAND[1] or BAND[0] <= cert.max_ratio <= BAND[1]
    if not border:
        assert cert.rank_one == ref["rank_one"], (what, cert.max_ratio, ref["max_ratio"])
        assert cert.feasible == ref["feasible"], what
        assert cert.certified == ref["certified"], (what, cert.xi, ref["xi"])
    # the bound and the rollout cost of one certified point agree with the
    # oracle's to the accuracy of the solve
    if cert.certified and ref["certified"]:
        assert abs(cert.lower_bound - ref["lower_bound"]) <= 1e-5 * (1 + abs(ref["lower_bound"])), what
        assert abs(cert.phat - ref["phat"]) <= 1e-5 * (1 + abs(ref["phat"])), what


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pendulum_batch_of_8_matches_oracle(precision):
    """Pendulum N = 10, the 8 seeded instances of the batch, solved together
    in one batched solver (FP64 eigensolver, or FP32 with the FP64 polish)."""
    S = lib()
    idx = list(range(8))
    refs = _refs("pendulum", idx)
    probs = wl.problem_batch("pendulum", 8, N=10)
    P = [S.Problem(p) for p in probs]
    prec = S.STROM_PREC_FP64 if precision == "fp64" else S.STROM_PREC_MIXED
    solver = S.Solver([q.relax() for q in P], tol=1e-6, maxiter=20000, precision=prec, check_every=50)
    assert solver.solve() == S.STROM_OK
    certs = solver.certify_batch(P)
    for i in idx:
        _check(S, solver.result(i), certs[i], refs[i], ("pendulum", precision, i))


def test_served_requests_match_oracle():
    """16 seeded pendulum requests (N = 10) served by continuous batching
    over 256 slots, mixed into 480 other requests so that they are admitted
    at different times and share the device with other work: each result
    against the oracle's reference."""
    S = lib()
    idx = list(range(16))
    refs = _refs("pendulum", idx)
    probs = wl.problem_batch("pendulum", 16, N=10)
    filler = wl.problem_batch("pendulum", 480, seed=wl.BASE_SEED + 100_000, N=10)
    P = [S.Problem(p) for p in probs]
    F = [S.Problem(p) for p in filler]
    batch = S.Batch(P[0].relax(), 256, tol=1e-6, maxiter=20000, precision=S.STROM_PREC_MIXED, check_every=40)
    tickets = {}
    fi = 0
    for i in idx:
        # 30 filler requests before each reference request
        for _ in range(30):
            batch.submit(F[fi].relax(), F[fi])
            fi += 1
        tickets[i] = batch.submit(P[i].relax(), P[i])
    out = {}
    for _ in range(100000):
        run, queued = batch.step(40)
        for i, t in tickets.items():
            if i not in out:
                o = batch.poll(t)
                if o is not None:
                    out[i] = o
        if len(out) == len(idx):
            break
        assert run > 0 or queued > 0
    for i in idx:
        res, cert, lat = out[i]
        assert cert is not None
        _check(S, res, cert, refs[i], ("served", i))


def test_cartpole_batch_of_8_matches_oracle():
    """Cart-pole N = 50, the seeded instances that have an oracle reference
    (of the first 8), one batched solver with the sparse factor of the
    y-solve and a shared tail, FP64 eigensolver. Its relaxation is not tight
    (lambda_2 / lambda_1 about 0.7: not certified, like the oracle's), and
    at KKT 1e-6 the objective is still about 1e-5 (relative) from the
    optimum, so this test solves to KKT 1e-7 to hold the 1e-6 objective bar."""
    S = lib()
    if not os.path.exists(REFS):
        pytest.skip("no oracle references (tests/golden/make_oracle_refs.py)")
    have = json.load(open(REFS)).get("cartpole", {})
    idx = [i for i in range(8) if str(i) in have]
    if not idx:
        pytest.skip("no cart-pole oracle references yet")
    refs = [have[str(i)] for i in idx]
    probs = wl.problem_batch("cartpole", 8, N=50)
    P = [S.Problem(probs[i]) for i in idx]
    solver = S.Solver([q.relax() for q in P], tol=1e-7, maxiter=12000, precision=S.STROM_PREC_FP64,
                      check_every=100, factor=S.STROM_FACTOR_SPARSE)
    assert solver.solve() == S.STROM_OK
    certs = solver.certify_batch(P)
    for k, i in enumerate(idx):
        _check(S, solver.result(k), certs[k], refs[k], ("cartpole", i))
