"""Full-size parity in the served launch configuration: 1024 pendulum
(N = 10) instances in one solver, which runs the y-solve over tiles of two
instances sharing the factor of cliques 2..N as the serving measurement
does; sampled instances are checked against the oracle one by one."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import workloads as wl
from oracle import relax as OR
from oracle import sgs_admm as OA

from gpu_common import assert_close, dev, host, lib, torch

pytestmark = pytest.mark.gpu

SAMPLE = (0, 1, 511, 1022, 1023)


def test_full_batch_ysolve_and_first_iteration_sampled():
    S = lib()
    rng = np.random.default_rng(31)
    probs = [wl.pendulum_problem(N=10, theta0=float(t)) for t in rng.uniform(-0.2, 0.2, 1024)]
    with ThreadPoolExecutor(8) as ex:
        P = list(ex.map(S.Problem, probs))
        sd = list(ex.map(lambda p: p.relax(), P))
    red = {i: OA.reduce(OR.relax(probs[i])) for i in SAMPLE}
    fp64 = S.Solver(sd, tol=1e-12, maxiter=1, precision=S.STROM_PREC_FP64, check_every=1)
    # y = (A_K A_K^T)^{-1} r_K for every instance at once
    r = rng.standard_normal(fp64.m_total)
    rd = dev(r)
    yd = torch.zeros_like(rd)
    fp64.kernel_solve(rd.data_ptr(), yd.data_ptr())
    y = host(yd)
    for i in SAMPLE:
        rr = red[i]
        _, ro = fp64.offsets(i)
        assert np.array_equal(fp64.kept_rows(i), rr.keep)
        got = y[ro:ro + rr.sdp.m]
        want = OA.YSolver(rr.A)(r[ro:ro + rr.sdp.m][rr.keep])
        assert np.all(got[~rr.keep] == 0.0)
        assert_close(got[rr.keep], want, 1e-10, what=("y", i))
    # the first iteration of Algorithm 1: FP64, and mixed precision (FP32 eigensolver)
    fp64.step(1)
    mixed = S.Solver(sd, tol=1e-12, maxiter=1, precision=S.STROM_PREC_MIXED, check_every=1)
    mixed.step(1)
    for i in SAMPLE:
        ref = OA.solve(red[i], OA.Options(tol=1e-12, maxiter=1))
        for sv, tol in ((fp64, 1e-9), (mixed, 1e-5)):
            X, Sg, _ = sv.state(i)
            assert_close(X, ref.X, tol, what=("X", i, tol))
            assert_close(Sg, ref.S, tol, floor=1.0, what=("S", i, tol))
