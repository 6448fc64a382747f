#!/usr/bin/env python3
"""Throughput of the STROM hot path on GB300: certified solves per second.

Workload: pendulum swing-up, horizon N = 10, dt = 0.1, start angle
theta0 ~ U(-0.2, 0.2) rad (seeded: request i uses seed 20240607 + i), served
by continuous batching over B solver slots. Every request runs the whole hot
path: row reduction + factorisation of A A^T for its slot (setup),
sGS-ADMM (Algorithm 1) until max(eta_p, eta_d, eta_g) <= 1e-6, and the
certificate (rank-1 test, rollout, valid lower bound, xi). One step = a fixed
number of iterations of the served batch (requests admitted and retired as
slots free up). A solve counts when it converged and its certificate was
computed.

  value : steady-state served throughput after the warm-up steps, requests
          queued before timing
  e2e   : the same batch continued, each step building (relaxation from
          polynomial data) and submitting its replacement requests inside the
          timed region and reading every result on the host
  plain : single instances one at a time with the FP64 eigensolver

Multi-GPU: replicas only (independent batches per rank, no collective on the
data path); value = certified solves of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "certified solves/s at KKT<=1e-6 (batched+served vs plain FP64); p50/p99 latency"
SEED = 20240607


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="strom", choices=["strom", "reference"])
    ap.add_argument("--slots", type=int, default=1024)
    ap.add_argument("--iters", type=int, default=800, help="sGS-ADMM iterations per step")
    ap.add_argument("--horizon", type=int, default=10)
    ap.add_argument("--maxiter", type=int, default=20000)
    ap.add_argument("--plain", type=int, default=8, help="instances timed in the plain FP64 single-instance form")
    ap.add_argument("--cpu-budget", type=float, default=25.0)
    ap.add_argument("--batch", type=int, default=0, help="cartpole / rigid workloads: instances (0 = 256 / 128)")
    ap.add_argument("--horizon-batch", type=int, default=0,
                    help="cartpole / rigid workloads: horizon (0 = 50 / N ~ U{20..100})")
    ap.add_argument("--check", type=int, default=100, help="cartpole / rigid workloads: iterations between checks")
    ap.add_argument("--eig-reorth", type=int, default=0,
                    help="cartpole / rigid workloads: re-orthonormalise the FP32 warm-start eigenvectors (0 / 1)")
    ap.add_argument("--workload", default="served", choices=["served", "psd", "warm", "poisson", "cartpole", "rigid",
                                                           "mixed"],
                    help="served: certified solves/s (default); psd: the 4096-block PSD-projection microbench; "
                         "warm: nearest-neighbour warm starts from a database of solved pendulums; "
                         "poisson: open-loop Poisson arrivals served cold and with warm starts from solved requests")
    ap.add_argument("--rate", type=float, default=40.0, help="poisson / mixed workloads: arrivals per second")
    ap.add_argument("--kinds", default="pendulum,cartpole", help="mixed workload: robots served")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="mixed workload: device-memory budget")
    ap.add_argument("--slots-class", type=int, default=64, help="mixed workload: most slots per structure")
    ap.add_argument("--drain", type=float, default=120.0, help="mixed workload: seconds served after the last arrival")
    ap.add_argument("--duration", type=float, default=12.0, help="poisson workload: seconds of arrivals")
    ap.add_argument("--step-iters", type=int, default=40, help="poisson workload: iterations per serving step")
    ap.add_argument("--warm-grid", type=int, default=9, help="warm workload: database grid points per key axis")
    ap.add_argument("--warm-queries", type=int, default=256, help="warm workload: batched queries")
    ap.add_argument("--warm-single", type=int, default=4, help="warm workload: single-instance FP64 queries")
    ap.add_argument("--profile", default="none", choices=["none", "iterations", "psd", "cartpole"],
                    help="run a few launches of one case and exit (for ncu captures); prints no JSON")
    ap.add_argument("--precision", type=int, default=1, help="psd workload / profile: 0 = FP64, 1 = FP32")
    ap.add_argument("--polish-eta", type=float, default=1e-6,
                    help="switch an instance to the FP64 eigensolver once eta <= this (FP32 before)")
    return ap.parse_args()


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return self.summarise(self.lines)

    @staticmethod
    def summarise(lines):
        """Median and maximum SM clock and the throttle reasons seen active in
        nvidia-smi CSV lines (the fields of Q, no header, no units)."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# workload
# --------------------------------------------------------------------------
def make_problems(B, N, offset):
    import workloads as wl
    return wl.problem_batch("pendulum", B, seed=SEED + offset, N=N)


def relax_all(S, problems):
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        P = list(ex.map(S.Problem, problems))
        sdps = list(ex.map(lambda p: p.relax(), P))
    return P, sdps


def chain_solve_flops(sdp, keep):
    """FP64 flops of one block-banded y-solve (forward + backward) of one instance.

    The triangular factors cover the rows kept by the row reduction that are
    not moment-duplication rows: per clique group of m rows, m (m + 1) / 2
    multiply-adds forward and again backward, plus the coupling with the
    previous group's c kept consensus rows (m c each way).
    """
    import numpy as np
    a = sdp.export()
    oth = (a.row_kind != 0) & keep
    flops = 0
    prev_c = 0
    for k in range(int(a.row_clique.max()) + 1):
        rows = oth & (a.row_clique == k)
        m = int(rows.sum())
        cons = int(np.sum((a.row_kind == 4) & (a.row_clique == k) & keep))
        flops += 2 * (m * (m + 1) + 2 * m * prev_c)
        prev_c = cons
    return flops


def psd_flops(sizes, r_frac=0.7):
    """W(n) = 9 n^3 + 2 n^2 r per block (symmetric eigendecomposition + recombination)."""
    return sum(9 * n ** 3 + 2 * n * n * (r_frac * n) for n in sizes)


class Feeder:
    """Seeded pendulum requests, relaxed by the library's builder in worker threads."""

    def __init__(self, S, N, seed0):
        self.S, self.N, self.next = S, N, seed0

    def take(self, k):
        import numpy as np
        import workloads as wl
        probs = []
        for i in range(k):
            rng = np.random.default_rng(np.random.PCG64(self.next + i))
            probs.append(wl.pendulum_problem(N=self.N, theta0=float(rng.uniform(-0.2, 0.2))))
        self.next += k
        return relax_all(self.S, probs)


def combine_ranks(dist, t, counts, device):
    """Whole-job timing over replicas: the slowest rank's time and the sum of every rank's counts.

    Replicas serve independent requests, so this host-side reduction is the
    only exchange between ranks (none on the data path).
    """
    import torch
    tt = torch.tensor([float(t)], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    cc = torch.tensor([float(c) for c in counts], device=device, dtype=torch.float64)
    dist.all_reduce(cc)
    return float(tt.item()), [int(round(c)) for c in cc.tolist()]


def run_e2e(S, batch, feed, per_step, steps, iters, stream, outstanding, harvest, sync):
    """Serving end to end through the public API: each step builds its
    replacement requests from polynomial data (relaxation), submits them,
    serves `iters` iterations and reads every finished result on the host.
    The requests of step k + 1 are built on a host thread while the GPU
    serves step k (the library calls release the interpreter lock).
    Returns (counted solves, seconds, transfer bytes before, after, tickets
    still outstanding)."""
    from concurrent.futures import ThreadPoolExecutor
    done = 0
    with ThreadPoolExecutor(max_workers=1) as prep:
        b0 = S.transfer_bytes()
        t0 = time.perf_counter()
        nxt = prep.submit(feed.take, per_step)
        for _ in range(steps):
            P, sd = nxt.result()
            outstanding += [batch.submit(x, pr) for x, pr in zip(sd, P)]
            del P, sd
            nxt = prep.submit(feed.take, per_step)
            batch.step(iters, stream)
            d, outstanding = harvest(outstanding)
            done += sum(1 for f in d if f[0].status == S.STROM_OK and f[1] is not None and f[1].xi == f[1].xi)
        sync()
        te = time.perf_counter() - t0
        b1 = S.transfer_bytes()
        del nxt   # requests prepared for a step that is not run
    return done, te, b0, b1, outstanding


def run_strom(a, rank, world):
    import numpy as np
    import torch
    import paper_2406_05846_gb300 as S

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    S.lib()
    B, N, it = a.slots, a.horizon, a.iters
    feed = Feeder(S, N, SEED + rank * 10_000_000)
    P0, sd0 = feed.take(1)
    opts = dict(tol=1e-6, maxiter=a.maxiter, precision=S.STROM_PREC_MIXED, polish_eta=a.polish_eta,
                check_every=a.iters)
    batch = S.Batch(sd0[0], B, **opts)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    # requests for the whole run, queued in host memory before timing (their
    # A, b, C values are uploaded at admission, inside the timed region)
    per_step = max(1, int(B * it / 1200))      # expected retirements per step (about 2000 iterations each)
    total = B + (a.warmup + a.steps + 1) * per_step
    outstanding = []
    while len(outstanding) < total:
        k = min(512, total - len(outstanding))
        P, sd = feed.take(k)
        outstanding += [batch.submit(x, pr) for x, pr in zip(sd, P)]
        del P, sd

    def harvest(tickets):
        done, keep = [], []
        for t in tickets:
            o = batch.poll(t, with_service=True)
            (keep if o is None else done).append(t if o is None else o)
        return done, keep

    for _ in range(a.warmup):
        batch.step(it, sp)
    _, outstanding = harvest(outstanding)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = Clocks(dev)
    clk.start()
    l0 = S.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    finished = []
    for _ in range(a.steps):
        batch.step(it, sp)
        d, outstanding = harvest(outstanding)
        finished += d
    e1.record(stream)
    torch.cuda.synchronize()
    launches = S.launch_count() - l0
    clocks = clk.stop()
    t = e0.elapsed_time(e1) / 1e3
    ok = [f for f in finished if f[0].status == S.STROM_OK and f[1] is not None and f[1].xi == f[1].xi]
    solved = len(ok)
    if dist:
        t, (solved,) = combine_ranks(dist, t, [solved], "cuda")
    value = solved / t
    svc = np.array([f[3] for f in ok]) if ok else np.array([np.nan])
    iters = np.array([f[0].iterations for f in ok]) if ok else np.array([0])
    cert_frac = float(np.mean([f[1].certified for f in ok])) if ok else 0.0
    verdicts = {"rank_one": sum(f[1].rank_one for f in ok), "rollout_feasible": sum(f[1].feasible for f in ok),
                "xi_le_1pct": sum(f[1].xi <= 1e-2 for f in ok), "certified": sum(f[1].certified for f in ok),
                "of": len(ok)}

    # ---- end to end through the public API, continuing the same warmed batch
    e2e_done, te, (h2d0, d2h0), (h2d1, d2h1), outstanding = run_e2e(
        S, batch, feed, per_step, a.steps, it, sp, outstanding, harvest, torch.cuda.synchronize)
    e2e = {"value": e2e_done / te, "unit": "solves/s", "h2d_bytes_per_step": (h2d1 - h2d0) // a.steps,
           "d2h_bytes_per_step": (d2h1 - d2h0) // a.steps}
    del batch

    # ---- the plain single-instance FP64 form on the same kind of requests
    # (the seeded instances 0.. of the pendulum batch, which have stored
    # oracle references: objective and verdict against the oracle)
    import workloads as wl
    plain_lat = []
    plain_ok = 0
    plain_par = []
    refs = _oracle_refs("pendulum")
    Pp, sdp = relax_all(S, wl.problem_batch("pendulum", a.plain, N=N))
    for i in range(a.plain):
        sv = S.Solver([sdp[i]], tol=1e-6, maxiter=a.maxiter, precision=S.STROM_PREC_FP64, check_every=100)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sv.factor()
        sv.solve()
        c = sv.certify(0, Pp[i])
        torch.cuda.synchronize()
        plain_lat.append(time.perf_counter() - t0)
        r = sv.result(0)
        plain_ok += r.status == S.STROM_OK
        ref = refs.get(str(i)) if N == 10 else None
        if ref is not None and r.status == S.STROM_OK:
            plain_par.append((abs(r.pobj - ref["pobj"]) / (1 + abs(ref["pobj"])), c.certified == ref["certified"]))
        del sv
    plain = {"value": plain_ok / sum(plain_lat) if plain_lat else None, "unit": "solves/s",
             "instances": a.plain, "precision": "fp64 eigensolver, fp64 y-solve", "mode": "one instance at a time",
             "latency_s": plain_lat, "latency_p50_s": float(np.median(plain_lat)) if plain_lat else None,
             "oracle_parity": {"instances": len(plain_par),
                               "max_rel_obj": max((p[0] for p in plain_par), default=None),
                               "verdicts_equal": sum(p[1] for p in plain_par)}}

    # ---- roofline of the dominant kernel, timed live on this stream
    Pr, sdr = feed.take(B)
    solver = S.Solver(sdr, **opts)
    roof = roofline(S, solver, sdr, stream)
    del solver
    cpu = cpu_baseline(a) if (rank == 0 and world == 1) else None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * t / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": "pendulum swing-up N=%d dt=0.1 (theta0~U(-0.2,0.2) seeded), served by continuous "
                                   "batching over %d slots, %d sGS-ADMM iterations per step, KKT<=1e-6, FP32 Jacobi "
                                   "eig, FP64 Jacobi polish once eta<=%g (retirement only on an FP64 iterate), "
                                   "FP64 y-solve, certificate per request" % (N, B, it, a.polish_eta),
                       "slots": B, "iters_per_step": it, "horizon": N, "maxiter": a.maxiter,
                       "inputs": "requests queued in host memory before timing; each admission uploads its A, b, C "
                                 "values and refactorises its slot inside the timed region",
                       "l2": "working set (about %.1f GB of slot state and factors) larger than L2" % (B * 9.0e-3),
                       "parallelism": "replicas x%d" % world},
            "e2e": e2e, "gpu_launches": launches,
            "latency_s": {"service_p50": float(np.percentile(svc, 50)), "service_p99": float(np.percentile(svc, 99)),
                          "plain_single_p50": float(np.median(plain_lat)) if plain_lat else None},
            "iterations": {"p50": float(np.percentile(iters, 50)), "p99": float(np.percentile(iters, 99))},
            "completed": len(finished), "counted": solved,
            "converged": sum(1 for f in finished if f[0].status == S.STROM_OK),
            "maxiter_hit": sum(1 for f in finished if f[0].status == S.STROM_MAXITER),
            "converged_fraction_of_completed": (sum(1 for f in finished if f[0].status == S.STROM_OK)
                                                / max(1, len(finished))),
            "certified_fraction": cert_frac,
            "rank1_certified_per_s": verdicts["certified"] / t, "verdicts": verdicts,
            "plain_fp64": plain, "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
        }
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def roofline(S, solver, sdps, stream):
    """Time the y-solve (FP64, chain kernel) and the FP32 projection live; report the larger one."""
    import numpy as np
    import torch
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    sp = stream.cuda_stream
    m, n = solver.m_total, solver.nsvec_total
    r = torch.randn(m, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(r)
    keep = [solver.kept_rows(i) for i in range(len(sdps))]
    f_solve = sum(chain_solve_flops(s, k) for s, k in zip(sdps, keep))
    reps = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    solver.kernel_solve(r.data_ptr(), y.data_ptr(), sp)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        solver.kernel_solve(r.data_ptr(), y.data_ptr(), sp)
    e1.record(stream)
    torch.cuda.synchronize()
    t_solve = e0.elapsed_time(e1) / 1e3 / reps
    # projection of every block of the batch in FP32 (the hot eigensolver)
    offs, ns = [], []
    for i, s in enumerate(sdps):
        a = s.export()
        so, _ = solver.offsets(i)
        offs.append(a.block_off + so)
        ns.append(a.block_n)
    offs, ns = np.concatenate(offs), np.concatenate(ns)
    plan = S.PsdPlan(offs, ns, S.STROM_PREC_FP32)
    x = torch.randn(n, dtype=torch.float64, device="cuda")
    o = torch.zeros_like(x)
    plan.execute(x.data_ptr(), o.data_ptr(), None, sp)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        plan.execute(x.data_ptr(), o.data_ptr(), None, sp)
    e1.record(stream)
    torch.cuda.synchronize()
    t_psd = e0.elapsed_time(e1) / 1e3 / reps
    f_psd = psd_flops(ns.tolist())
    # ALU peaks from unit counts and the maximum SM clock: SMs x 2 FP64
    # (128 FP32) FMA per clock x 2 flops x clock; an FMA-loop probe on this
    # part measured 1.208 and 75.49 TFLOP/s
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    fp64_peak = sms * 2 * 2 * clk / 1e12
    fp32_peak = sms * 128 * 2 * clk / 1e12
    # the method's own work for the same solves: the sparse Cholesky factor
    # of the star-eliminated system (strom_sdp_factor_info), 2 flops per
    # stored entry forward and again backward
    fi_cache = {}
    for sd in sdps:
        k = (sd.m, sd.nsvec)
        if k not in fi_cache:
            fi = sd.factor_info()
            fi_cache[k] = 4 * fi["nnz_L"] + 4 * fi["n_other"]
    f_sparse = sum(fi_cache[(sd.m, sd.nsvec)] for sd in sdps)
    # DRAM bytes (read + write) of one y-solve launch over 1024 pendulum
    # (N = 10) instances, from an ncu capture of the unchanged kernel
    traffic = 1.708e9 + 39.6e6 if (len(sdps) == 1024 and sdps[0].info.N == 10) else None
    if solver.factor_kind == S.STROM_FACTOR_SPARSE:
        traffic = None   # the capture above is of the dense kernel
    sparse = solver.factor_kind == S.STROM_FACTOR_SPARSE
    if sparse:
        f_solve = f_sparse   # the sparse factor's own work
    if 2 * t_solve >= t_psd:
        ach = f_solve / t_solve / 1e12
        if sparse:
            kname = "sp_solve_kernel (sparse factor, block substitution)"
        else:
            kname = ("chain_solve_multi_kernel<2> (dense per-clique groups, tiles of 2 instances sharing the "
                     "factor of cliques 2..N)" if len(sdps) >= 304 else "chain_solve_kernel (dense per-clique groups)")
        return {"kernel": "chain y-solve, FP64: " + kname, "bound": "alu", "achieved": ach,
                "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak, "traffic": traffic,
                "peak_basis": "%d SMs x 2 FP64 FMA/clk x %.2f GHz (FMA-loop probe: 1.208 TFLOP/s FP64)"
                              % (sms, clk / 1e9),
                "method_work": {"flops_per_launch": f_sparse, "achieved": f_sparse / t_solve / 1e12,
                                "frac": f_sparse / t_solve / 1e12 / fp64_peak,
                                "basis": "sparse Cholesky factor of the star-eliminated system (4 flops per "
                                         "stored entry per solve): the work the method needs"},
                "launch_ms": 1e3 * t_solve, "other": {"jacobi_psd_fp32_ms": 1e3 * t_psd,
                                                      "jacobi_psd_fp32_tflops": f_psd / t_psd / 1e12}}
    ach = f_psd / t_psd / 1e12
    return {"kernel": "jacobi_psd_kernel (FP32)", "bound": "alu", "achieved": ach, "peak": fp32_peak,
            "unit": "TFLOP/s", "frac": ach / fp32_peak, "traffic": None, "launch_ms": 1e3 * t_psd,
            "other": {"chain_solve_ms": 1e3 * t_solve, "chain_solve_tflops": f_solve / t_solve / 1e12}}


def _cpu_worker(q, horizon, budget, maxiter, offset):
    import numpy as np  # noqa: F401
    import workloads as wl
    from oracle import certify as OC
    from oracle import relax as OR
    from oracle import sgs_admm as OA
    t0 = time.perf_counter()
    done = 0
    tried = 0
    i = offset
    while time.perf_counter() - t0 < budget or tried == 0:
        p = wl.problem_batch("pendulum", i + 1, seed=SEED, N=horizon)[i]
        red = OA.reduce(OR.relax(p))
        res = OA.solve(red, OA.Options(tol=1e-6, maxiter=maxiter))
        if res.converged:
            OC.certify(p, red, res.X, res.y)
            done += 1
        tried += 1
        i += 1
    q.put((done, tried, time.perf_counter() - t0))


def _oracle_sample(a, budget, offset):
    """The oracle worker in a spawned single-threaded process: (converged, tried, seconds)."""
    import multiprocessing as mp
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        pr = ctx.Process(target=_cpu_worker, args=(q, a.horizon, budget, a.maxiter, offset))
        pr.start()
        done, tried, t = q.get()
        pr.join()
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return done, tried, t


def cpu_baseline(a, budget=None, offset=0):
    """The FP64 oracle on one host core, on a bounded sample of the same workload."""
    budget = a.cpu_budget if budget is None else budget
    done, tried, t = _oracle_sample(a, budget, offset)
    return {"value": done / t, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": "%d pendulum N=%d instances (seeded, from instance %d) solved to KKT<=1e-6 and certified "
                      "by the FP64 NumPy/SciPy oracle in %.1f s on one core (%d converged)"
                      % (tried, a.horizon, offset, t, done)}


def run_reference(a, rank, world):
    """The reference arm: the FP64 CPU oracle, one seeded instance per step, on one host core."""
    if rank != 0:
        return
    runs = [_oracle_sample(a, 1e-9, k) for k in range(a.warmup + a.steps)][a.warmup:]
    done = sum(r[0] for r in runs)
    tot = sum(r[2] for r in runs)
    value = done / tot if tot > 0 else 0.0
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot / max(1, a.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "pendulum swing-up N=%d dt=0.1, one instance per step (theta0~U(-0.2,0.2) seeded), "
                                   "KKT<=1e-6, FP64 CPU oracle" % a.horizon, "horizon": a.horizon,
                       "maxiter": a.maxiter},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": "%d instances, one per step, FP64 oracle on one core (%d converged)"
                                       % (a.steps, done)},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_profile(a):
    """A few launches of one case, for ncu: 3 sGS-ADMM iterations on a batch of
    `--slots` pendulum instances, or 3 projections of the microbench."""
    import torch
    import paper_2406_05846_gb300 as S
    S.lib()
    if a.profile == "iterations":
        feed = Feeder(S, a.horizon, SEED)
        _, sd = feed.take(a.slots)
        sv = S.Solver(sd, tol=1e-6, precision=a.precision, check_every=1)
        sv.step(3)
    elif a.profile == "cartpole":
        import workloads as wl
        _, sd = relax_all(S, wl.problem_batch("cartpole", a.batch or 256, N=a.horizon_batch or 50))
        sv = S.Solver(sd, tol=1e-6, precision=S.STROM_PREC_MIXED, check_every=10, factor=S.STROM_FACTOR_SPARSE)
        sv.step(30)
    else:
        import workloads as wl
        x, off, n, _ = wl.psd_microbench()
        xb = torch.tensor(x, device="cuda")
        o = torch.zeros_like(xb)
        plan = S.PsdPlan(off, n, a.precision)
        for _ in range(3):
            plan.execute(xb.data_ptr(), o.data_ptr())
    torch.cuda.synchronize()


def run_psd(a):
    """The PSD-projection microbench: 4096 blocks {8: 40%, 36: 30%, 78: 20%,
    136: 10%} with prescribed spectra, FP64 svec in and out (blocks/s)."""
    import numpy as np
    import torch
    import paper_2406_05846_gb300 as S
    import workloads as wl
    from oracle import jacobi as OJ
    from oracle import relax as OR
    S.lib()
    x, off, n, _ = wl.psd_microbench()
    xb = torch.tensor(x, device="cuda")
    o = torch.zeros_like(xb)
    plan = S.PsdPlan(off, n, a.precision)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    for _ in range(a.warmup):
        plan.execute(xb.data_ptr(), o.data_ptr(), None, sp)
    torch.cuda.synchronize()
    clk = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    l0 = S.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        plan.execute(xb.data_ptr(), o.data_ptr(), None, sp)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = S.launch_count() - l0
    t = e0.elapsed_time(e1) / 1e3 / a.steps
    got = o.cpu().numpy()
    # sampled parity against the oracle's LAPACK-free cyclic Jacobi projection
    # (8 blocks of each size)
    rng = np.random.default_rng(0)
    err = 0.0
    for k in (8, 36, 78, 136):
        for b in rng.choice(np.nonzero(n == k)[0], 8, replace=False):
            tt = k * (k + 1) // 2
            X = OR.smat(x[off[b]:off[b] + tt], k)
            err = max(err, np.linalg.norm(OR.smat(got[off[b]:off[b] + tt], k) - OJ.project_block(X))
                      / np.linalg.norm(X))
    # end to end: host svec in, host svec out
    h = torch.tensor(x).pin_memory()
    ho = torch.empty_like(h).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        xb.copy_(h, non_blocking=True)
        plan.execute(xb.data_ptr(), o.data_ptr(), None, sp)
        ho.copy_(o, non_blocking=True)
        torch.cuda.synchronize()
    te = (time.perf_counter() - t0) / a.steps
    flops = psd_flops(n.tolist())
    fp = 152 * (128 if a.precision == 1 else 2) * 2 * 2.07e9 / 1e12   # unit counts x 2.07 GHz
    line = {"metric": "PSD projections per second (4096-block microbench)", "value": len(n) / t, "unit": "blocks/s",
            "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if a.precision == 1 else "f64",
            "data": "synthetic",
            "config": {"workload": "4096 symmetric blocks {8:40%,36:30%,78:20%,136:10%}, spectra 1e-4..1 with 30% "
                                   "negative, Haar eigenvectors, seed 1", "l2": "inputs 58 MB (fit in L2)"},
            "e2e": {"value": len(n) / te, "unit": "blocks/s", "h2d_bytes_per_step": int(8 * len(x)),
                    "d2h_bytes_per_step": int(8 * len(x))},
            "gpu_launches": launches, "max_rel_error_vs_oracle": err,
            "roofline": {"kernel": "jacobi_psd_kernel", "bound": "alu", "achieved": flops / t / 1e12, "peak": fp,
                         "unit": "TFLOP/s", "frac": flops / t / 1e12 / fp, "traffic": None,
                         "algorithmic_flops": flops},
            "clocks": clocks}
    print(json.dumps(line))


def _oracle_refs(kind):
    """The FP64 oracle's stored reference solves (tests/golden/oracle_refs.json,
    written by tests/golden/make_oracle_refs.py from oracle/ alone)."""
    try:
        return json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_refs.json"))).get(kind, {})
    except OSError:
        return {}


def run_batch(a):
    """One batched solve of many instances in one solver (configs 3 and 4):
    the cart-pole swing-up x256 at N = 50, or the planar rigid body x128 with
    horizons N ~ U{20..100} and 2-4 disk obstacles. FP32 Jacobi eigensolver
    with the FP64 polish, FP64 sparse factor of the y-solve. A step is the
    whole solve: set-up from device-resident data (row reduction,
    factorisation), Algorithm 1 until every instance met KKT <= 1e-6 or
    maxiter, certificates. Reported: certified solves/s, the time at which
    each instance was seen converged (p50/p99, checked every check_every
    iterations), and the objectives of the instances that have an oracle
    reference."""
    import numpy as np
    import torch
    import paper_2406_05846_gb300 as S
    import workloads as wl
    S.lib()
    kind = "cartpole" if a.workload == "cartpole" else "rigid_body"
    B = a.batch or (256 if kind == "cartpole" else 128)
    kw = {"N": a.horizon_batch or 50} if kind == "cartpole" else ({"N": a.horizon_batch} if a.horizon_batch else {})
    probs = wl.problem_batch(kind, B, **kw)
    t0 = time.perf_counter()
    P, sdps = relax_all(S, probs)
    t_relax = time.perf_counter() - t0
    opts = dict(tol=1e-6, maxiter=a.maxiter, precision=S.STROM_PREC_MIXED, polish_eta=a.polish_eta,
                check_every=a.check, factor=S.STROM_FACTOR_SPARSE, eig_reorth=a.eig_reorth)
    t0 = time.perf_counter()
    sv = S.Solver(sdps, **opts)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    for _ in range(a.warmup):     # graph capture, module loading, first-touch
        sv.step(a.check, sp)
    torch.cuda.synchronize()
    clk = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    l0 = S.launch_count()
    e0, e1, ef = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    t0 = time.perf_counter()
    e0.record(stream)
    sv.factor(sp)
    ef.record(stream)
    seen = np.full(B, np.nan)
    done_it = 0
    while done_it < a.maxiter:
        act = sv.step(a.check, sp)
        done_it += a.check
        now = time.perf_counter() - t0
        for i in np.nonzero(np.isnan(seen))[0]:
            if sv.result(int(i)).status != S.STROM_MAXITER or act == 0:
                seen[i] = now
        if act == 0:
            break
    certs = sv.certify_batch(P)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    t_setup = e0.elapsed_time(ef) / 1e3
    clocks = clk.stop()
    launches = S.launch_count() - l0
    res = [sv.result(i) for i in range(B)]
    conv = [r.status == S.STROM_OK for r in res]
    # a certified solve: converged at KKT <= 1e-6 with its certificate
    # computed (whatever its verdict: the cart-pole's relaxation is not tight)
    ok = [c and cert is not None and cert.xi == cert.xi for c, cert in zip(conv, certs)]
    rank1 = [c and cert.certified for c, cert in zip(conv, certs)]
    iters = np.array([r.iterations for r in res])
    lat = seen[np.array(conv)] if any(conv) else np.array([np.nan])
    refs = _oracle_refs(kind)
    parity = []
    for i in range(B):
        ref = refs.get(str(i)) if kind == "cartpole" else next(
            (v for v in refs.values() if v["index"] == i), None)
        if ref is None or not ref.get("converged") or not conv[i]:
            continue
        parity.append({"i": i, "rel_obj": abs(res[i].pobj - ref["pobj"]) / (1 + abs(ref["pobj"])),
                       "verdict_equal": bool(certs[i].certified == ref["certified"])})
    Ns = [p.N for p in probs]
    line = {"metric": METRIC, "value": sum(ok) / t, "unit": "solves/s", "n_gpus": 1, "steps": 1,
            "warmup": a.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": ("cart-pole swing-up x%d, N=%d, dt=0.05 (x0~U(-0.5,0.5), theta0~U(-0.3,0.3) "
                                    "seeded)" % (B, Ns[0])) if kind == "cartpole" else
                       ("planar rigid body x%d, N in [%d, %d] (mean %.1f), 2-4 disks seeded" %
                        (B, min(Ns), max(Ns), float(np.mean(Ns)))),
                       "instances": B, "maxiter": a.maxiter, "check_every": a.check,
                       "precision": "FP32 Jacobi eig, FP64 polish once eta<=%g, FP64 sparse y-solve factor"
                                    % a.polish_eta,
                       "inputs": "resident in HBM; the step re-runs the set-up (row reduction, factorisation) "
                                 "from device data"},
            "completed": B, "converged": int(sum(conv)), "maxiter_hit": int(sum(r.status == S.STROM_MAXITER
                                                                            for r in res)),
            "counted": int(sum(ok)), "rank1_certified": int(sum(rank1)), "gpu_launches": launches,
            "seconds": {"relax_host": t_relax, "solver_create": t_create, "setup_in_step": t_setup, "step": t},
            "latency_s": {"converged_p50": float(np.percentile(lat, 50)),
                          "converged_p99": float(np.percentile(lat, 99))},
            "iterations": {"p50": float(np.percentile(iters, 50)), "p99": float(np.percentile(iters, 99)),
                           "max": int(iters.max())},
            "oracle_parity": {"instances": len(parity),
                              "max_rel_obj": max((p["rel_obj"] for p in parity), default=None),
                              "verdicts_equal": sum(p["verdict_equal"] for p in parity)},
            "clocks": clocks}
    print(json.dumps(line))


def solve_status(S, sv):
    """strom_solve, keeping the per-instance statuses when one instance hit NaN/Inf."""
    from paper_2406_05846_gb300._native import StromError
    try:
        return sv.solve()
    except StromError as e:
        if e.status != -4:
            raise
        return e.status


def run_warm(a):
    """Data-driven warm starts (Sec. 5, inverted pendulum): a database of
    solved pendulums on a grid of initial states (theta0, omega0) in
    [-0.2, 0.2] x [-0.5, 0.5], solved offline by this solver; new initial
    states (seeded, uniform over the same box) start from the convex
    combination of their nearest stored solutions. Reported: throughput and
    iterations of the same queries solved cold and warm (batched), and the
    latency of single instances in the plain FP64 form."""
    import numpy as np
    import torch
    import paper_2406_05846_gb300 as S
    import workloads as wl
    S.lib()
    N, G, Q = a.horizon, a.warm_grid, a.warm_queries
    scale = np.array([0.2, 0.5])
    opts = dict(tol=1e-6, maxiter=a.maxiter, precision=S.STROM_PREC_MIXED, polish_eta=a.polish_eta, check_every=50)

    def relax(params):
        P = [wl.pendulum_problem(N=N, theta0=float(t), omega0=float(w)) for t, w in params]
        return relax_all(S, P)

    grid = [(t, w) for t in np.linspace(-0.2, 0.2, G) for w in np.linspace(-0.5, 0.5, G)]
    Pg, sdg = relax(grid)
    t0 = time.perf_counter()
    dbs = S.Solver(sdg, **opts)
    solve_status(S, dbs)
    db_time = time.perf_counter() - t0
    store = S.WarmStore(2, sdg[0].nsvec, len(grid))
    stored = 0
    for i, p in enumerate(grid):
        if dbs.result(i).status == S.STROM_OK:
            store.add_from_solver(dbs, i, np.array(p) / scale)
            stored += 1
    del dbs
    rng = np.random.default_rng(np.random.PCG64(SEED + 777))
    queries = np.column_stack([rng.uniform(-0.2, 0.2, Q), rng.uniform(-0.5, 0.5, Q)])
    Pq, sdq = relax(queries)
    stream = torch.cuda.current_stream()
    clk = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    out = {}
    for mode in ("cold", "warm"):
        sv = S.Solver(sdq, **opts)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if mode == "warm":
            for i, q in enumerate(queries):
                sv.warm_start(i, store, q / scale)
        solve_status(S, sv)
        certs = sv.certify_batch(Pq)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        res = [sv.result(i) for i in range(Q)]
        ok = [r.status == S.STROM_OK for r in res]
        it = np.array([r.iterations for r in res])
        bad = [[float(queries[i][0]), float(queries[i][1])] for i, r in enumerate(res) if r.status < 0]
        out[mode] = {"solves_per_s": sum(ok) / t, "time_s": t, "converged": int(sum(ok)), "numerical": bad,
                     "certified": int(sum(c.certified for c in certs)),
                     "iterations_p50": float(np.percentile(it, 50)), "iterations_p99": float(np.percentile(it, 99)),
                     "iterations_max": int(it.max()), "pobj": [r.pobj for r in res], "ok": ok}
        del sv
    pc, pw = np.array(out["cold"].pop("pobj")), np.array(out["warm"].pop("pobj"))
    both = np.array(out["cold"].pop("ok")) & np.array(out["warm"].pop("ok"))
    objdiff = float(np.max(np.abs(pw - pc)[both] / (1 + np.abs(pc[both]))))
    # single instances, plain FP64 form, one at a time
    single = {"cold": [], "warm": []}
    iters1 = {"cold": [], "warm": []}
    for i in range(min(a.warm_single, Q)):
        for mode in ("cold", "warm"):
            sv = S.Solver([sdq[i]], tol=1e-6, maxiter=a.maxiter, precision=S.STROM_PREC_FP64, check_every=50)
            torch.cuda.synchronize()
            ts = time.perf_counter()
            if mode == "warm":
                sv.warm_start(0, store, queries[i] / scale)
            solve_status(S, sv)
            sv.certify(0, Pq[i])
            torch.cuda.synchronize()
            single[mode].append(time.perf_counter() - ts)
            iters1[mode].append(sv.result(0).iterations)
            del sv
    clocks = clk.stop()
    line = {"metric": "certified solves/s with nearest-neighbour warm starts (pendulum N=%d)" % N,
            "value": out["warm"]["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": True, "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": "pendulum swing-up N=%d dt=0.1, initial state (theta0, omega0) ~ U([-0.2,0.2] x "
                                   "[-0.5,0.5]) seeded, %d queries solved in one batch, KKT<=1e-6, certificate "
                                   "per query; warm start = convex combination of the stored solutions of the "
                                   "nearest database states (barycentric in their triangle)" % (N, Q),
                       "database": "%dx%d grid over the same box, solved by this solver (%d converged, %.1f s)"
                                   % (G, G, stored, db_time),
                       "key_scale": scale.tolist()},
            "cold": out["cold"], "warm": out["warm"], "speedup_batched": out["warm"]["solves_per_s"] /
            max(1e-12, out["cold"]["solves_per_s"]), "objective_max_rel_diff_warm_vs_cold": objdiff,
            "single_fp64": {"cold_latency_s": single["cold"], "warm_latency_s": single["warm"],
                            "cold_iterations": iters1["cold"], "warm_iterations": iters1["warm"]},
            "clocks": clocks}
    print(json.dumps(line))


def run_poisson(a):
    """Open-loop serving: pendulum requests (N=10, (theta0, omega0) uniform in
    [-0.2, 0.2] x [-0.5, 0.5]) arrive as a seeded Poisson process of rate
    --rate for --duration seconds and are served by continuous batching.
    Run twice on the same arrivals: cold starts, and warm starts from the
    nearest requests already solved (each converged request is recorded in a
    device-resident store keyed by its initial state; the store starts
    empty). Latency = arrival to the host seeing the result, queueing
    included."""
    import numpy as np
    import torch
    import paper_2406_05846_gb300 as S
    import workloads as wl
    S.lib()
    N = a.horizon
    scale = np.array([0.2, 0.5])
    rng = np.random.default_rng(np.random.PCG64(SEED + 4242))
    gaps = rng.exponential(1.0 / a.rate, size=int(a.rate * a.duration * 2) + 16)
    arr = np.cumsum(gaps)
    arr = arr[arr < a.duration]
    n = arr.size
    keys = np.column_stack([rng.uniform(-0.2, 0.2, n), rng.uniform(-0.5, 0.5, n)])
    P, sd = relax_all(S, [wl.pendulum_problem(N=N, theta0=float(t), omega0=float(w)) for t, w in keys])
    opts = dict(tol=1e-6, maxiter=a.maxiter, precision=S.STROM_PREC_MIXED, polish_eta=a.polish_eta,
                check_every=a.step_iters)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    clk = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    out = {}
    for mode in ("cold", "warm"):
        batch = S.Batch(sd[0], a.slots, **opts)
        store = None
        if mode == "warm":
            store = S.WarmStore(2, sd[0].nsvec, n)
            batch.set_warm(store, record=True)
        pending = {}
        lat, its, cert, ok = [], [], 0, 0
        nxt = 0
        drain = a.duration + 45.0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while True:
            now = time.perf_counter() - t0
            while nxt < n and arr[nxt] <= now:
                if mode == "warm":
                    t = batch.submit_keyed(sd[nxt], keys[nxt] / scale, P[nxt])
                else:
                    t = batch.submit(sd[nxt], P[nxt])
                pending[t] = nxt
                nxt += 1
            if not pending and nxt >= n:
                break
            if now > drain:
                break
            if pending:
                batch.step(a.step_iters, sp)
            else:
                time.sleep(max(0.0, min(0.01, arr[nxt] - now)))
            done_at = time.perf_counter() - t0
            for t in list(pending):
                o = batch.poll(t)
                if o is None:
                    continue
                j = pending.pop(t)
                res, c, _ = o
                if res.status == S.STROM_OK:
                    ok += 1
                    lat.append(done_at - arr[j])
                    its.append(res.iterations)
                    cert += bool(c is not None and c.certified)
        span = time.perf_counter() - t0
        lat, its = np.array(lat or [np.nan]), np.array(its or [0])
        out[mode] = {"arrived": int(n), "converged": ok, "certified": cert, "unfinished": len(pending),
                     "solves_per_s": ok / span, "span_s": span,
                     "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                     "iterations_p50": float(np.percentile(its, 50)), "iterations_p99": float(np.percentile(its, 99)),
                     "store_entries": len(store) if store is not None else 0}
        del batch, store
    clocks = clk.stop()
    line = {"metric": "served pendulum requests under Poisson arrivals: latency (arrival to result) and solves/s",
            "value": out["warm"]["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": True, "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": "pendulum swing-up N=%d, (theta0, omega0) ~ U([-0.2,0.2] x [-0.5,0.5]) seeded, "
                                   "Poisson arrivals %.0f/s for %.0f s (%d requests), %d slots, %d iterations per "
                                   "serving step, KKT<=1e-6, certificate per request" %
                                   (N, a.rate, a.duration, n, a.slots, a.step_iters),
                       "warm": "each converged request is recorded (key = initial state); a new request starts "
                               "from the combination of its nearest recorded solutions; store empty at start"},
            "cold": out["cold"], "warm": out["warm"], "clocks": clocks}
    print(json.dumps(line))


def serving_case(j, kind, converged, certified, pobj, ref):
    """One sampled served request against the oracle's solve of it at the
    served accuracy (KKT 1e-6, the same iteration limit): it passes when
    both reach the same outcome, converged with the same verdict or both
    stopped at the iteration limit."""
    return {"request": j, "kind": kind, "converged": converged, "oracle_converged": ref["converged"],
            "rel_obj": abs(pobj - ref["pobj"]) / (1 + abs(ref["pobj"])),
            "certified": certified, "oracle_certified": ref["certified"],
            "pass": converged == ref["converged"] and (not converged or certified == ref["certified"])}


def run_mixed(a):
    """Serving the mixed stream (50% pendulum N ~ U{10..60}, 30% cart-pole
    N ~ U{20..80}, 20% planar rigid body N ~ U{20..100}; seeded) arriving as a
    Poisson process of rate --rate for --duration seconds, through one
    strom_server: one batch per structure class, sized from an HBM byte
    budget (--budget-gb), idle batches evicted when another structure needs
    the room, every batch with work stepped at once. --kinds restricts the
    robots (requests of other robots are dropped from the same stream).
    Latency = arrival to the host seeing the result, queueing included. The
    requests that have a stored oracle reference (tests/golden/oracle_refs.json,
    set "mixed", keyed by request index) are compared with it."""
    import numpy as np
    import torch
    import paper_2406_05846_gb300 as S
    import workloads as wl
    S.lib()
    kinds = set(a.kinds.split(","))
    arr_all = wl.poisson_arrivals(a.rate, a.duration)
    reqs = []
    for j, t in enumerate(arr_all):
        kind, p = wl.mixed_request(j)
        if kind in kinds:
            reqs.append((j, t, kind, p))
    P, sd = relax_all(S, [r[3] for r in reqs])
    opts = dict(tol=1e-6, maxiter=a.maxiter, precision=S.STROM_PREC_MIXED, polish_eta=a.polish_eta,
                check_every=a.step_iters)
    srv = S.Server(int(a.budget_gb * 1e9), a.slots_class, **opts)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    clk = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    refs = _oracle_refs("mixed")
    pending, res = {}, {}
    nxt = 0
    l0 = S.launch_count()
    torch.cuda.synchronize()
    clk.start()
    t0 = time.perf_counter()
    limit = a.duration + a.drain
    while True:
        now = time.perf_counter() - t0
        while nxt < len(reqs) and reqs[nxt][1] <= now:
            pending[srv.submit(sd[nxt], P[nxt])] = nxt
            nxt += 1
        if (not pending and nxt >= len(reqs)) or now > limit:
            break
        if pending:
            srv.step(a.step_iters, sp)
        else:
            time.sleep(max(0.0, min(0.01, reqs[nxt][1] - now)))
        done_at = time.perf_counter() - t0
        for t in list(pending):
            o = srv.poll(t)
            if o is not None:
                k = pending.pop(t)
                res[k] = (o, done_at - reqs[k][1])
    span = time.perf_counter() - t0
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = S.launch_count() - l0
    classes, used = srv.info()
    per = {}
    for kind in sorted(kinds):
        ks = [k for k in range(len(reqs)) if reqs[k][2] == kind]
        ok = [k for k in ks if k in res and res[k][0][0].status == S.STROM_OK]
        lat = np.array([res[k][1] for k in ok] or [np.nan])
        its = np.array([res[k][0][0].iterations for k in ok] or [0])
        per[kind] = {"arrived": len(ks), "converged": len(ok),
                     "maxiter": sum(1 for k in ks if k in res and res[k][0][0].status == S.STROM_MAXITER),
                     "unfinished": sum(1 for k in ks if k not in res),
                     "certified": sum(1 for k in ok if res[k][0][1] is not None and res[k][0][1].certified),
                     "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                     "iterations_p50": float(np.percentile(its, 50))}
    ok_all = [k for k in res if res[k][0][0].status == S.STROM_OK]
    lat = np.array([res[k][1] for k in ok_all] or [np.nan])
    parity = []
    for k, (j, _, kind, _) in enumerate(reqs):
        ref = refs.get(str(j))
        if ref is None or k not in res:
            continue
        r, c = res[k][0][0], res[k][0][1]
        parity.append(serving_case(j, kind, r.status == S.STROM_OK, bool(c is not None and c.certified), r.pobj,
                                   ref))
    line = {"metric": "served mixed requests under Poisson arrivals: solves/s, latency (arrival to result)",
            "value": len(ok_all) / span, "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": True, "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": "mixed stream (pendulum N~U{10..60} 50%%, cart-pole N~U{20..80} 30%%, rigid body "
                                   "N~U{20..100} 20%%; robots served: %s), Poisson %.1f/s for %.0f s, %d requests "
                                   "served, budget %.0f GB, at most %d slots per structure, %d iterations per step, "
                                   "KKT<=1e-6, certificate per request" %
                                   (",".join(sorted(kinds)), a.rate, a.duration, len(reqs), a.budget_gb,
                                    a.slots_class, a.step_iters)},
            "span_s": span, "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "per_robot": per, "classes": len(classes), "budget_used_gb": used / 1e9,
            "batches_created": sum(c["batches_created"] for c in classes), "gpu_launches": launches,
            "oracle_parity": {"sampled": len(parity),
                              "both_converged": sum(p["converged"] and p["oracle_converged"] for p in parity),
                              "max_rel_obj_both_converged": max((p["rel_obj"] for p in parity
                                                                 if p["converged"] and p["oracle_converged"]),
                                                                default=None),
                              "pass_rate": (sum(p["pass"] for p in parity) / len(parity)) if parity else None,
                              "cases": parity},
            "clocks": clocks}
    print(json.dumps(line))


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    if a.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit("bench.py --gpus %d: launch one process per GPU with torch.distributed.run "
                 "(--nproc-per-node %d); a single process measures one GPU" % (a.gpus, a.gpus))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if a.profile != "none":
        run_profile(a)
    elif a.impl == "reference":
        run_reference(a, rank, world)
    elif a.workload == "psd":
        run_psd(a)
    elif a.workload == "warm":
        run_warm(a)
    elif a.workload == "poisson":
        run_poisson(a)
    elif a.workload in ("cartpole", "rigid"):
        run_batch(a)
    elif a.workload == "mixed":
        run_mixed(a)
    else:
        run_strom(a, rank, world)


if __name__ == "__main__":
    main()
