"""Writes tests/golden/oracle_refs.json: the FP64 oracle's reference solves of
the seeded instances that the whole-solve GPU parity tests compare against.

Each reference is Algorithm 1 of the oracle (oracle/sgs_admm.py) run to
max(eta_p, eta_d, eta_g) <= 1e-8 (the objective parity of a GPU solve at
1e-6 is judged against it), followed by the oracle's certificate
(oracle/certify.py: rank-1 test, extraction, rollout, lower bound, xi) at
that solution. Only oracle/ computes; workloads/ supplies the seeded inputs.

Sets (instance i of a set is workloads.problem_batch(kind, ...)[i]):
  pendulum    N = 10, seeds 0..15 of the pendulum batch (0..7: batched solves;
              all 16: requests of a served batch)
  cartpole    N = 50, seeds 0..7 of the cart-pole batch
  rigid_body  the 8 instances of the 128-instance uneven batch
              (N ~ U{20..100}) with the shortest horizons
  mixed       requests of the seeded serving stream (workloads.mixed_request,
              keyed by request index): the first 16 pendulum requests and the
              first 6 cart-pole requests, solved at the served accuracy
              (KKT 1e-6, at most 20,000 iterations, as the server): at these
              horizons Algorithm 1 can stall far above 1e-8 (the pendulum at
              N = 31 and 52 stood at eta_d ~ 4e-4 and 8e-4 after 60,000
              iterations)

Usage: python tests/golden/make_oracle_refs.py SET [SET ...] [--workers K]
Existing entries are kept; only missing ones are computed. Single-threaded BLAS per worker.
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "oracle_refs.json")

RIGID_BATCH = 128
TOL = 1e-8
MAXITER = 60000


def instances(kind):
    sys.path.insert(0, ROOT)
    import workloads as wl
    if kind == "pendulum":
        ps = wl.problem_batch("pendulum", 16, N=10)
        return [(i, p) for i, p in enumerate(ps)]
    if kind == "cartpole":
        ps = wl.problem_batch("cartpole", 8, N=50)
        return [(i, p) for i, p in enumerate(ps)]
    if kind == "rigid_body":
        ps = wl.problem_batch("rigid_body", RIGID_BATCH)
        order = sorted(range(len(ps)), key=lambda i: (ps[i].N, i))[:8]
        return [(i, ps[i]) for i in sorted(order)]
    if kind == "mixed":
        out, npend, ncart = [], 0, 0
        for j in range(10000):
            k, p = wl.mixed_request(j)
            if k == "pendulum" and npend < 16:
                out.append((j, p))
                npend += 1
            elif k == "cartpole" and ncart < 6:
                out.append((j, p))
                ncart += 1
            if npend == 16 and ncart == 6:
                return out
    raise ValueError(kind)


def solve_one(args):
    kind, i = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    sys.path.insert(0, ROOT)
    from oracle import certify as OC
    from oracle import relax as OR
    from oracle import sgs_admm as OA
    p = dict(instances(kind))[i]
    t0 = time.time()
    red = OA.reduce(OR.relax(p))
    tol, maxiter = (1e-6, 20000) if kind == "mixed" else (TOL, MAXITER)
    res = OA.solve(red, OA.Options(tol=tol, maxiter=maxiter))
    c = OC.certify(p, red, res.X, res.y)
    return {"kind": kind, "index": i, "N": p.N, "robot": p.name, "tol": tol, "maxiter": maxiter,
            "iterations": res.iters, "converged": bool(res.converged),
            "pobj": res.pobj, "dobj": res.dobj, "eta": [res.eta_p, res.eta_d, res.eta_g],
            "m_kept": int(red.keep.sum()), "max_ratio": c.max_ratio, "feasible": bool(c.feasible),
            "rank_one": bool(c.rank_one), "certified": bool(c.certified), "lower_bound": c.lower_bound,
            "phat": c.phat, "xi": c.xi, "seconds": time.time() - t0}


def main(argv):
    workers = 4
    if "--workers" in argv:
        k = argv.index("--workers")
        workers = int(argv[k + 1])
        argv = argv[:k] + argv[k + 2:]
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    refs = json.load(open(OUT)) if os.path.exists(OUT) else {}
    jobs = [(kind, i) for kind in argv for i, _ in instances(kind) if str(i) not in refs.get(kind, {})]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        for r in pool.imap_unordered(solve_one, jobs):
            # re-read before each write: entries another run added meanwhile are kept
            refs = json.load(open(OUT)) if os.path.exists(OUT) else {}
            refs.setdefault(r["kind"], {})[str(r["index"])] = r
            tmp = "%s.%d.tmp" % (OUT, os.getpid())
            with open(tmp, "w") as f:
                json.dump(refs, f, indent=1, sort_keys=True)
            os.replace(tmp, OUT)
            print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
